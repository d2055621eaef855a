"""TDI with nested delay operators (tdi_nested = 1, Sec. II.B delays applied
as products of one-link operators): the FP64 and mixed GPU paths against the
oracle's nested form, the GPU's nested-minus-summed difference against the
oracle's, laser-noise cancellation through the GPU TDI kernel, and logL."""
import math

import numpy as np
import pytest

from oracle import likelihood, orbits, pipeline, response
from paper_2501_08261_gb300 import api, workloads

from helpers import gpu_kwargs, norm_rel, oracle_setup

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

torch = pytest.importorskip("torch")
LINKS = (1, 2, 3, -1, -2, -3)


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2501_08261_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _lik(cfg, W, precision=0):
    return api.Likelihood(precision=precision, max_walkers=W, **gpu_kwargs(cfg))


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _smooth_links(n, W, seed):
    rng = np.random.default_rng(seed)
    y = np.zeros((6, n, W))
    for w in range(W):
        for j in range(6):
            y[j, :, w] = np.convolve(rng.normal(size=n), np.hanning(25), mode="same")
    return y


def _oracle_aet(y, w, cfg, s, nested):
    yd = {l: y[j, :, w] for j, l in enumerate(LINKS)}
    X, Y, Z = response.tdi_xyz(yd, cfg["n"], 0.0, cfg["dt"], s.orbit, cfg["tdi_gen"], 31,
                               nested=nested)
    return np.stack(response.aet_from_xyz(X, Y, Z))


@pytest.mark.parametrize("gen", [15, 20])
def test_nested_tdi_fp64_matches_oracle(gen):
    cfg = workloads.config("c1_fp64_1d", tdi_gen=gen, orbit=1, n=4320, tdi_nested=1)
    s = oracle_setup(cfg)
    W = 3
    y = _smooth_links(cfg["n"], W, 5)
    got = _lik(cfg, W).tdi(_t(y)).cpu().numpy()
    summed = _lik(dict(cfg, tdi_nested=0), W).tdi(_t(y)).cpu().numpy()
    for w in range(W):
        want = _oracle_aet(y, w, cfg, s, True)
        want_sum = _oracle_aet(y, w, cfg, s, False)
        for c in range(3):
            assert norm_rel(got[c, :, w], want[c]) < 1e-10, (w, c)
            # the nested form moves the delays by ~1e-7 s; the GPU reproduces
            # the oracle's change, not just its own summed result
            d_gpu = got[c, :, w] - summed[c, :, w]
            d_orc = want[c] - want_sum[c]
            assert np.max(np.abs(d_orc)) > 1e-9 * np.max(np.abs(want[c]))
            assert np.max(np.abs(d_gpu - d_orc)) <= 2e-2 * np.max(np.abs(d_orc)), (w, c)


def test_nested_tdi_mixed_matches_oracle():
    cfg = workloads.config("c1_fp64_1d", tdi_gen=20, orbit=1, n=4320, tdi_nested=1)
    s = oracle_setup(cfg)
    W = 70
    y = _smooth_links(cfg["n"], W, 6)
    got = _lik(cfg, W, precision=1).tdi(_t(y, torch.float32)).cpu().numpy()
    for w in (0, 33, 64, 69):
        want = _oracle_aet(y, w, cfg, s, True)
        for c in range(3):
            assert norm_rel(got[c, :, w], want[c]) < 1e-4, (w, c)


def test_nested_tdi_cancels_laser_noise_on_gpu():
    """One laser per craft, y_l(t) = p_s(t - L_l(t)) - p_r(t) on the grid: the
    GPU's TDI 2 with nested operators removes it to the FP64 rounding of the
    samples; the summed delays leave the first-order arm-rate term."""
    cfg = workloads.config("c1_fp64_1d", tdi_gen=20, orbit=1, n=4320, tdi_nested=1)
    n, dt = cfg["n"], cfg["dt"]
    t = np.arange(n) * dt
    rng = np.random.default_rng(12)
    lasers = {k: [(rng.uniform(0.5, 1.0), rng.uniform(1e-3, 2e-2), rng.uniform(0, 2 * math.pi))
                  for _ in range(4)] for k in (1, 2, 3)}

    def p(k, u):                      # laser k at t + u (angle addition about t)
        out = 0.0
        for (a, f, ph) in lasers[k]:
            base = 2 * math.pi * f * t + ph
            out = out + a * (np.sin(base) * np.cos(2 * math.pi * f * u)
                             + np.cos(base) * np.sin(2 * math.pi * f * u))
        return out

    y = np.zeros((6, n, 1))
    for j, l in enumerate(LINKS):
        s_, r_ = orbits.LINK_ENDS[l]
        y[j, :, 0] = p(s_, -orbits.light_time("kepler", l, t)) - p(r_, np.zeros(n))
    inner = slice(48, n - 24)          # stencils inside the grid
    nested = _lik(cfg, 1).tdi(_t(y)).cpu().numpy()[:, inner, 0]
    summed = _lik(dict(cfg, tdi_nested=0), 1).tdi(_t(y)).cpu().numpy()[:, inner, 0]
    r_n, r_s = np.max(np.abs(nested)), np.max(np.abs(summed))
    assert r_s > 1e-9
    assert r_n < 1e-10 and r_n < 1e-3 * r_s, (r_n, r_s)


def _snr_scaled(truth, s, snr):
    d = pipeline.aet(truth, s)
    rho = math.sqrt(-2 * likelihood.loglike(np.zeros_like(d), d, s.dt, s.f_lo, s.f_hi,
                                            s.tdi_gen, s.channel_mask))
    th = truth.copy()
    th[8] *= rho / snr
    return th, d * (snr / rho)


def test_nested_loglike_fp64_and_mixed():
    cfg = workloads.config("c2_hm_1d", n=8640, tdi_gen=20, orbit=1, tdi_nested=1)
    s = oracle_setup(cfg)
    truth = workloads.prior_draws(1, cfg["n"], cfg["dt"], 31, logm=(5.5, 7.0))[0]
    truth, d = _snr_scaled(truth, s, 2000.0)
    z = workloads.standard_normals(5, 15, 32)
    th = np.repeat(truth[None], 6, axis=0)
    for w in range(1, 6):
        th[w, 11] += 2e-4 * z[w - 1, 0]
        th[w, 12] += 2e-4 * z[w - 1, 1]
        th[w, 14] += 0.2 * z[w - 1, 2]
    want = np.array([pipeline.loglike(x, s, d) for x in th])
    for precision in (0, 1):
        lk = _lik(cfg, 6, precision)
        lk.set_data(_t(d))
        got = lk.loglike(_t(th)).cpu().numpy()
        for g, o in zip(got, want):
            bar = max(1e-6, 1e-11 * abs(o)) if precision == 0 else max(0.05, 1e-4 * abs(o))
            assert abs(g - o) <= bar, (precision, g, o)


def test_nested_full_size_sampled_outputs():
    cfg = workloads.config("c2_hm_60d", tdi_nested=1)
    s = oracle_setup(cfg)
    th = workloads.prior_draws(2, cfg["n"], cfg["dt"], 61, logm=(5.5, 7.0))
    lk = _lik(cfg, 2, precision=1)
    aet = lk.tdi(lk.project(_t(th))).cpu().numpy()
    idx = np.unique(np.concatenate([np.arange(0, 40), np.arange(cfg["n"] - 40, cfg["n"]),
                                    np.random.default_rng(4).integers(0, cfg["n"], 160)]))
    for w in range(2):
        want = pipeline.aet(th[w], s, idx=idx)
        scale = np.max(np.abs(aet[:, :, w]))
        for c in range(3):
            assert np.max(np.abs(aet[c, idx, w] - want[c])) <= 1e-4 * scale, (w, c)
