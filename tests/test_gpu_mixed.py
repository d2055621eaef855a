"""Parity of the mixed-precision GPU path (FP32 arithmetic, double-float
phase/time, FP64 anchors) with the FP64 oracle.  Bars: 1e-4 norm-relative on
series; |dlogL| <= max(0.05, 1e-4 |logL|) at SNR 2000 -- 0.05 absolute for the
posterior bulk, 1e-4 relative for far walkers (|logL| >> 500, where 0.05 is
below FP32 resolution)."""
import math

import numpy as np
import pytest

from oracle import likelihood, pipeline, response
from paper_2501_08261_gb300 import api, workloads

from helpers import gpu_kwargs, norm_rel, oracle_setup

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]
torch = pytest.importorskip("torch")
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2501_08261_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _lik(cfg, W):
    return api.Likelihood(precision=1, max_walkers=W, **gpu_kwargs(cfg))


def _walkers(cfg, w, seed):
    return workloads.prior_draws(w, cfg["n"], cfg["dt"], seed,
                                 precessing=bool(cfg["precessing"]), logm=(5.5, 7.0))


CONFIGS = ["c1_fp64_1d", "c2_hm_1d", "c3_prec_1d"]


@pytest.mark.parametrize("name", CONFIGS)
def test_mixed_waveform(name):
    cfg = workloads.config(name)
    th = _walkers(cfg, 3, 11)
    h = _lik(cfg, 3).waveform(_t(th)).cpu().numpy()
    s = oracle_setup(cfg)
    bar = 1e-4 if cfg["precessing"] else 1e-5   # precession angles partly in FP32
    for w in range(3):
        hp, hc = pipeline.polarizations(th[w], s)
        assert norm_rel(h[w, :, 0], hp) < bar, w
        assert norm_rel(h[w, :, 1], hc) < bar, w


@pytest.mark.parametrize("name", CONFIGS)
def test_mixed_projection(name):
    cfg = workloads.config(name)
    th = _walkers(cfg, 2, 12)
    y = _lik(cfg, 2).project(_t(th)).cpu().numpy()
    s = oracle_setup(cfg)
    for w in range(2):
        hp, _ = pipeline.polarizations(th[w], s)
        yo = pipeline.links(th[w], s)
        for j, l in enumerate((1, 2, 3, -1, -2, -3)):
            # y is a difference of two interpolated h values: its rounding error
            # scales with |h|, so the bar is relative to max(|y|, 1e-2 |h|)
            scale = max(np.max(np.abs(yo[l])), 1e-2 * np.max(np.abs(hp)))
            assert np.max(np.abs(y[j, :, w] - yo[l])) <= TOL * scale, (w, l)


# dt = 5 s runs the kernel with one combined FIR per (channel, link); at
# dt = 1 s the terms of a pair spread over more than 64 taps, so the kernel
# with one FIR per term runs
@pytest.mark.parametrize("gen,orbit,dt", [(15, 0, 5.0), (20, 1, 5.0), (15, 0, 1.0), (20, 1, 1.0)])
def test_mixed_tdi_of_oracle_links(gen, orbit, dt):
    cfg = workloads.config("c1_fp64_1d", tdi_gen=gen, orbit=orbit, n=4320, dt=dt)
    s = oracle_setup(cfg)
    rng = np.random.default_rng(5)
    W = 70                                        # two CTA walker blocks, ragged
    y = np.zeros((6, cfg["n"], W))
    for w in range(W):
        for j in range(6):
            y[j, :, w] = np.convolve(rng.normal(size=cfg["n"]), np.hanning(25), mode="same")
    aet = _lik(cfg, W).tdi(torch.as_tensor(y, dtype=torch.float32, device="cuda")).cpu().numpy()
    for w in (0, 1, 33, 63, 64, 69):
        yd = {l: y[j, :, w] for j, l in enumerate((1, 2, 3, -1, -2, -3))}
        X, Y, Z = response.tdi_xyz(yd, cfg["n"], 0.0, cfg["dt"], s.orbit, gen, 31)
        want = response.aet_from_xyz(X, Y, Z)
        for c in range(3):
            assert norm_rel(aet[c, :, w], want[c]) < TOL, (w, c)


def _snr_scaled(truth, s, snr):
    d = pipeline.aet(truth, s)
    rho = math.sqrt(-2 * likelihood.loglike(np.zeros_like(d), d, s.dt, s.f_lo, s.f_hi,
                                            s.tdi_gen, s.channel_mask))
    th = truth.copy()
    th[8] *= rho / snr
    return th, d * (snr / rho)


@pytest.mark.parametrize("name", CONFIGS)
def test_mixed_loglike_bulk_and_far(name):
    cfg = workloads.config(name)
    s = oracle_setup(cfg)
    truth = _walkers(cfg, 1, 21)[0]
    truth, d = _snr_scaled(truth, s, 2000.0)
    z = workloads.standard_normals(8, 15, 23)
    th = np.repeat(truth[None], 9, axis=0)
    scales = {8: 2e-3, 11: 2e-4, 12: 2e-4, 14: 0.2, 0: 2e-5, 9: 1e-3, 13: 1e-3}
    for w in range(1, 9):
        for p, sc in scales.items():
            th[w, p] += (sc * z[w - 1, p] * th[w, p]) if p in (0, 8) else sc * z[w - 1, p]
    th[8, 12] += 0.05                              # a far walker
    lk = _lik(cfg, 9)
    lk.set_data(_t(d))
    got = lk.loglike(_t(th)).cpu().numpy()
    want = np.array([pipeline.loglike(t, s, d) for t in th])
    for g, o in zip(got, want):
        assert abs(g - o) <= max(0.05, 1e-4 * abs(o)), (g, o)
    assert abs(got[0]) <= 0.05


@pytest.mark.parametrize("name", ["c2_hm_60d", "c3_prec_60d"])
def test_mixed_full_size_sampled_outputs(name):
    cfg = workloads.config(name)
    s = oracle_setup(cfg)
    th = _walkers(cfg, 2, 60)
    lk = _lik(cfg, 2)
    aet = lk.tdi(lk.project(_t(th))).cpu().numpy()
    idx = np.unique(np.concatenate([np.arange(0, 40), np.arange(cfg["n"] - 40, cfg["n"]),
                                    np.random.default_rng(3).integers(0, cfg["n"], 220)]))
    for w in range(2):
        want = pipeline.aet(th[w], s, idx=idx)
        scale = np.max(np.abs(aet[:, :, w]))
        for c in range(3):
            assert np.max(np.abs(aet[c, idx, w] - want[c])) <= TOL * scale, (w, c)


def test_mixed_matches_fp64_gpu_at_bench_shape():
    """60 d, 5 mode pairs, Keplerian TDI-2, 64 walkers: mixed vs FP64 GPU logL
    (both against the same injection at SNR ~ 2000)."""
    cfg = workloads.config("c2_hm_60d")
    W = 64
    th = _walkers(cfg, W, 70)
    lk64 = api.Likelihood(precision=0, max_walkers=W, **gpu_kwargs(cfg))
    lk32 = _lik(cfg, W)
    s = oracle_setup(cfg)
    truth, d = _snr_scaled(th[0], s, 2000.0)
    th[0] = truth
    th[1:8] = truth
    th[1:8, 14] += np.linspace(-1.0, 1.0, 7)       # bulk walkers near the injection
    for lk in (lk64, lk32):
        lk.set_data(_t(d))
    a = lk64.loglike(_t(th)).cpu().numpy()
    b = lk32.loglike(_t(th)).cpu().numpy()
    for g, o in zip(b, a):
        assert abs(g - o) <= max(0.05, 1e-4 * abs(o)), (g, o)


def test_bench_configuration_256_walkers_autotuned():
    """The configuration bench.py times: 60 d, 256 walkers, the mixed context
    autotuned for them (lisa_td_autotune), an SNR-2000 injection.  Walkers
    1..64 are the posterior bulk: draws from N(theta_inj, F^-1) in all eleven
    parameters of the aligned source (F from the FP64 likelihood) whose FP64
    logL is >= -100, at least 32 of them.  logL of all
    256 walkers against the FP64 GPU path (0.05 absolute on the bulk, relative
    1e-4 for far walkers), and sampled A, E, T outputs of the injection walker
    in the tuned launch shapes against the oracle."""
    from paper_2501_08261_gb300 import mcmc
    cfg = workloads.config("c2_hm_60d")
    W = 256
    th = _walkers(cfg, W, 71)
    s = oracle_setup(cfg)
    truth, d = _snr_scaled(th[0], s, 2000.0)
    th[0] = truth
    lk64 = api.Likelihood(precision=0, max_walkers=W, **gpu_kwargs(cfg))
    lk64.set_data(_t(d))
    ball = mcmc.fisher_ball(lk64, truth, mcmc.ALIGNED_IDX, 128, seed=72)
    keep = torch.nonzero(lk64.loglike(ball) >= -100.0).flatten()[:64].cpu().numpy()
    assert len(keep) >= 32, len(keep)                    # a posterior-bulk set of >= 32
    th[1:1 + len(keep)] = ball.cpu().numpy()[keep]
    nb = 1 + len(keep)
    a = lk64.loglike(_t(th)).cpu().numpy()
    lk64.close()
    lk32 = _lik(cfg, W)
    lk32.set_data(_t(d))
    choice = api.lisa_td_autotune(lk32.ctx, _t(th), W)
    b = lk32.loglike(_t(th)).cpu().numpy()
    for w, (g, o) in enumerate(zip(b, a)):
        assert abs(g - o) <= max(0.05, 1e-4 * abs(o)), (w, choice, g, o)
    assert np.max(np.abs(b[:nb] - a[:nb])) <= 0.05
    idx = np.unique(np.concatenate([np.arange(0, 24), np.arange(cfg["n"] - 24, cfg["n"]),
                                    np.random.default_rng(5).integers(0, cfg["n"], 120)]))
    aet = lk32.tdi(lk32.project(_t(th[:1]))).cpu().numpy()[:, :, 0]
    want = pipeline.aet(th[0], s, idx=idx)
    scale = np.max(np.abs(aet))
    for c in range(3):
        assert np.max(np.abs(aet[c, idx] - want[c])) <= TOL * scale, (c, choice)
    lk32.close()
