"""Parity of the FP64 GPU path with the FP64 oracle, stage by stage and end to
end, through the C ABI.  Tolerances: 1e-10 norm-relative on series, 1e-6
absolute (or 1e-11 relative for |logL| > 1e5) on logL."""
import math

import numpy as np
import pytest

from oracle import likelihood, pipeline, response, waveform
from paper_2501_08261_gb300 import api, workloads

from helpers import gpu_kwargs, norm_rel, oracle_setup

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

torch = pytest.importorskip("torch")
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2501_08261_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _walkers(cfg, w, seed):
    pts = workloads.prior_draws(w, cfg["n"], cfg["dt"], seed, precessing=bool(cfg["precessing"]),
                                logm=(5.5, 7.0))
    return pts


def _lik(cfg, W, precision=0):
    return api.Likelihood(precision=precision, max_walkers=W, **gpu_kwargs(cfg))


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


CONFIGS = ["c1_fp64_1d", "c2_hm_1d", "c3_prec_1d"]


@pytest.mark.parametrize("name", CONFIGS)
def test_waveform_matches_oracle(name):
    cfg = workloads.config(name)
    th = _walkers(cfg, 3, 11)
    lk = _lik(cfg, 3)
    h = lk.waveform(_t(th)).cpu().numpy()
    s = oracle_setup(cfg)
    for w in range(3):
        hp, hc = pipeline.polarizations(th[w], s)
        assert norm_rel(h[w, :, 0], hp) < TOL, w
        assert norm_rel(h[w, :, 1], hc) < TOL, w


@pytest.mark.parametrize("name", CONFIGS)
def test_projection_matches_oracle(name):
    cfg = workloads.config(name)
    th = _walkers(cfg, 2, 12)
    lk = _lik(cfg, 2)
    y = lk.project(_t(th)).cpu().numpy()
    s = oracle_setup(cfg)
    for w in range(2):
        hp, _ = pipeline.polarizations(th[w], s)
        yo = pipeline.links(th[w], s)
        for j, l in enumerate((1, 2, 3, -1, -2, -3)):
            # y = G (h(t_s) - h(t_r)) nearly cancels for slow signals (|y| can be
            # 1e-4 |h|); its FP64 rounding scales with |h|, hence the bar
            # relative to max(|y|, 1e-2 |h|)
            scale = max(np.max(np.abs(yo[l])), 1e-2 * np.max(np.abs(hp)))
            assert np.max(np.abs(y[j, :, w] - yo[l])) <= TOL * scale, (w, l)


@pytest.mark.parametrize("gen,orbit", [(15, 0), (20, 0), (15, 1), (20, 1)])
def test_tdi_of_oracle_links_matches_oracle(gen, orbit):
    cfg = workloads.config("c1_fp64_1d", tdi_gen=gen, orbit=orbit, n=4320)
    s = oracle_setup(cfg)
    rng = np.random.default_rng(5)
    W = 3
    y = np.zeros((6, cfg["n"], W))
    for w in range(W):
        for j in range(6):
            y[j, :, w] = np.convolve(rng.normal(size=cfg["n"]), np.hanning(25), mode="same")
    lk = _lik(cfg, W)
    aet = lk.tdi(_t(y)).cpu().numpy()
    for w in range(W):
        yd = {l: y[j, :, w] for j, l in enumerate((1, 2, 3, -1, -2, -3))}
        X, Y, Z = response.tdi_xyz(yd, cfg["n"], 0.0, cfg["dt"], s.orbit, gen, 31)
        want = response.aet_from_xyz(X, Y, Z)
        for c in range(3):
            assert norm_rel(aet[c, :, w], want[c]) < TOL, (w, c)


def _check_logl(got, want):
    for g, o in zip(got, want):
        assert abs(g - o) <= max(1e-6, 1e-11 * abs(o)), (g, o)


@pytest.mark.parametrize("name", CONFIGS)
def test_loglike_matches_oracle(name):
    cfg = workloads.config(name)
    s = oracle_setup(cfg)
    truth = _walkers(cfg, 1, 21)[0]
    d = pipeline.aet(truth, s)
    z = workloads.standard_normals(4, 15, 22)
    th = np.repeat(truth[None], 5, axis=0)
    th[1:, 11] += 1e-3 * z[:, 0]           # small sky / mass / time offsets
    th[1:, 12] += 1e-3 * z[:, 1]
    th[1:, 0] *= 1 + 1e-4 * z[:, 2]
    th[1:, 14] += 5.0 * z[:, 3]
    lk = _lik(cfg, 5)
    lk.set_data(_t(d))
    got = lk.loglike(_t(th)).cpu().numpy()
    want = [pipeline.loglike(t, s, d) for t in th]
    assert got[0] == pytest.approx(0.0, abs=1e-6)
    _check_logl(got, want)


def test_loglike_channel_masks_and_orders():
    for mask, p in ((1, 1), (3, 7), (5, 15)):
        cfg = workloads.config("c2_hm_1d", n=8640, channel_mask=mask, lagrange_order=p)
        s = oracle_setup(cfg)
        th = _walkers(cfg, 3, 30 + mask)
        d = pipeline.aet(th[0], s)
        lk = _lik(cfg, 3)
        lk.set_data(_t(d))
        got = lk.loglike(_t(th)).cpu().numpy()
        _check_logl(got, [pipeline.loglike(t, s, d) for t in th])


def test_ragged_walker_count_and_invalid_walkers():
    cfg = workloads.config("c1_fp64_1d", n=4320)
    s = oracle_setup(cfg)
    W = 37                                   # two walker groups, ragged tail
    th = _walkers(cfg, W, 40)
    d = pipeline.aet(th[0], s)
    th[5, 0] = np.nan
    th[9, 8] = -1.0
    lk = _lik(cfg, 64)
    lk.set_data(_t(d))
    got, st = lk.loglike(_t(th), with_status=True)
    got, st = got.cpu().numpy(), st.cpu().numpy()
    assert st[5] == 1 and st[9] == 1 and got[5] == -math.inf and got[9] == -math.inf
    assert np.all(st[[0, 1, 36]] == 0)
    idx = [0, 1, 17, 31, 32, 36]
    _check_logl(got[idx], [pipeline.loglike(th[i], s, d) for i in idx])


def test_single_walker_and_zero_distance_limit():
    cfg = workloads.config("c1_fp64_1d", n=2880)
    s = oracle_setup(cfg)
    th = _walkers(cfg, 1, 50)
    d = pipeline.aet(th[0], s)
    lk = _lik(cfg, 1)
    lk.set_data(_t(d))
    far = th.copy()
    far[0, 8] = 1e30                           # h -> 0: logL = -1/2 (d|d)
    dd = -2 * likelihood.loglike(np.zeros_like(d), d, s.dt, s.f_lo, s.f_hi, s.tdi_gen)
    got = lk.loglike(_t(far)).cpu().numpy()[0]
    assert got == pytest.approx(-0.5 * dd, rel=1e-12)


@pytest.mark.parametrize("name", ["c2_hm_60d", "c3_prec_60d"])
def test_full_size_sampled_outputs(name):
    """60 days, 2 walkers: AET at 300 sampled indices (oracle evaluated sparsely)."""
    cfg = workloads.config(name)
    s = oracle_setup(cfg)
    th = _walkers(cfg, 2, 60)
    lk = _lik(cfg, 2)
    y = lk.project(_t(th))
    aet = lk.tdi(y).cpu().numpy()
    idx = np.unique(np.concatenate([np.arange(0, 40), np.arange(cfg["n"] - 40, cfg["n"]),
                                    np.random.default_rng(3).integers(0, cfg["n"], 220)]))
    for w in range(2):
        want = pipeline.aet(th[w], s, idx=idx)
        scale = np.max(np.abs(aet[:, :, w]))
        for c in range(3):
            assert np.max(np.abs(aet[c, idx, w] - want[c])) <= TOL * scale, (w, c)
