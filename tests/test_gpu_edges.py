"""Edge cases of the batched likelihood: a thousand walkers (ragged tail of the
64-walker TDI groups), the smallest grids, and the mixed path at every
Lagrange order, each against the FP64 oracle or the FP64 GPU path."""
import numpy as np
import pytest

from oracle import pipeline
from paper_2501_08261_gb300 import api, workloads

from helpers import gpu_kwargs, oracle_setup

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2501_08261_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_thousand_walkers_mixed_vs_fp64_and_oracle():
    cfg = workloads.config("c2_hm_1d")
    W = 1000
    th = workloads.prior_draws(W, cfg["n"], 5.0, 81, logm=(5.5, 7.0))
    s = oracle_setup(cfg)
    d = pipeline.aet(th[0], s)
    far = th[0].copy()
    far[8] = 1e30
    rho = np.sqrt(-2.0 * pipeline.loglike(far, s, d))
    d = d * (2000.0 / rho)                      # the |dlogL| <= 0.05 bar holds at SNR <= 2000
    th[0, 8] *= rho / 2000.0
    l64 = api.Likelihood(precision=0, max_walkers=W, **gpu_kwargs(cfg))
    l32 = api.Likelihood(precision=1, max_walkers=W, **gpu_kwargs(cfg))
    l64.set_data(_t(d))
    l32.set_data(_t(d))
    a = l64.loglike(_t(th)).cpu().numpy()
    b = l32.loglike(_t(th)).cpu().numpy()
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(b))
    assert np.all(np.abs(a - b) <= np.maximum(0.05, 1e-4 * np.abs(a)))
    for w in (0, 511, 999):                     # first, a middle and the last (tail) walker
        o = pipeline.loglike(th[w], s, d)
        assert abs(a[w] - o) <= max(1e-6, 1e-11 * abs(o)), (w, a[w], o)
    l64.close()
    l32.close()


@pytest.mark.parametrize("n", [128, 640])
def test_small_grids_match_oracle(n):
    # grids shorter than the TDI halos and a light time: zero extension everywhere
    cfg = workloads.config("c1_fp64_1d", n=n)
    th = workloads.prior_draws(3, n, 5.0, 82, logm=(5.0, 5.5))
    th[:, 14] = 0.9 * n * 5.0
    s = oracle_setup(cfg)
    d = pipeline.aet(th[0], s)
    lk = api.Likelihood(precision=0, max_walkers=3, **gpu_kwargs(cfg))
    lk.set_data(_t(d))
    got = lk.loglike(_t(th)).cpu().numpy()
    for w in range(3):
        o = pipeline.loglike(th[w], s, d)
        assert abs(got[w] - o) <= max(1e-6, 1e-11 * abs(o)), (w, got[w], o)
    lk.close()


@pytest.mark.parametrize("p", [1, 3, 5, 7, 15])
def test_mixed_path_at_each_lagrange_order(p):
    cfg = workloads.config("c2_hm_1d", n=8640, lagrange_order=p)
    s = oracle_setup(cfg)
    th = workloads.prior_draws(4, cfg["n"], 5.0, 83 + p, logm=(5.5, 7.0))
    d = pipeline.aet(th[0], s)
    # the injection at SNR 500, three walkers near it and one far away
    far = th[0].copy()
    far[8] = 1e30
    rho = np.sqrt(-2.0 * pipeline.loglike(far, s, d))
    d = d * (500.0 / rho)
    th[0, 8] *= rho / 500.0
    th[1:3] = th[0]
    th[1, 14] += 2.0
    th[2, 11] += 1e-3
    lk = api.Likelihood(precision=1, max_walkers=4, **gpu_kwargs(cfg))
    lk.set_data(_t(d))
    got = lk.loglike(_t(th)).cpu().numpy()
    for w in range(4):
        o = pipeline.loglike(th[w], s, d)
        assert abs(got[w] - o) <= max(0.05, 1e-4 * abs(o)), (p, w, got[w], o)
    lk.close()


def _edge_walkers(base, precessing, n, dt):
    """The method's degenerate cases around one source: the bodies given in
    the wrong order (m2 > m1, the swap rule), the merger before the grid
    starts and after it ends, face-on and face-off inclinations, and for
    precessing spins no spin on body 1 and tilts of 0 and pi (beta -> 0, pi,
    the limits of the quaternion Wigner-D)."""
    out, names = [base.copy()], ["base"]

    def add(name, **kv):
        w = base.copy()
        for k, v in kv.items():
            w[int(k[1:])] = v
        out.append(w)
        names.append(name)
    add("m2>m1", p0=base[1], p1=base[0], p2=base[5], p3=base[6], p4=base[7],
        p5=base[2], p6=base[3], p7=base[4])
    add("merger_before_t0", p14=-600.0)
    add("merger_after_end", p14=n * dt + 3.0 * 3600.0)
    add("iota=0", p9=0.0)
    add("iota=pi", p9=np.pi)
    if precessing:
        add("a1=0", p2=0.0)
        add("tilt1=0", p3=0.0)
        add("tilt1=pi", p3=np.pi)
        add("both_tilts_pi", p3=np.pi, p6=np.pi)
    return np.array(out), names


@pytest.mark.parametrize("name", ["c2_hm_1d", "c3_prec_1d"])
@pytest.mark.parametrize("precision", [0, 1])
def test_degenerate_cases_match_oracle(name, precision):
    cfg = workloads.config(name)
    prec = bool(cfg["precessing"])
    s = oracle_setup(cfg)
    base = workloads.prior_draws(1, cfg["n"], cfg["dt"], 91, precessing=prec,
                                 logm=(5.8, 6.3))[0]
    th, names = _edge_walkers(base, prec, cfg["n"], cfg["dt"])
    d = pipeline.aet(base, s)
    far = base.copy()
    far[8] = 1e30
    rho = np.sqrt(-2.0 * pipeline.loglike(far, s, d))
    d = d * (500.0 / rho)
    th[:, 8] *= rho / 500.0
    W = th.shape[0]
    lk = api.Likelihood(precision=precision, max_walkers=W, **gpu_kwargs(cfg))
    lk.set_data(_t(d))
    got, st = lk.loglike(_t(th), with_status=True)
    got, st = got.cpu().numpy(), st.cpu().numpy()
    assert np.all(st == 0), dict(zip(names, st))
    for w in range(W):
        o = pipeline.loglike(th[w], s, d)
        tol = max(1e-6, 1e-11 * abs(o)) if precision == 0 else max(0.05, 1e-4 * abs(o))
        assert abs(got[w] - o) <= tol, (names[w], got[w], o)
    # the swap rule: the same binary with its bodies listed the other way round
    assert abs(got[1] - got[0]) <= (1e-9 if precision == 0 else 1e-3) * max(1.0, abs(got[0]))
    lk.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_grid_starting_a_year_later_matches_oracle(precision):
    """A grid that starts at t0 = one sidereal year plus 40 days (the
    constellation elsewhere on its orbit, and absolute times of 3.5e7 s, where
    FP32 resolves only 2 s): the mixed path carries time relative to t0 and
    FP64 anchors, so its logL must still meet the bars."""
    t0 = 31558149.763545603 + 40 * 86400.0
    cfg = workloads.config("c2_hm_1d", t0=t0)
    s = oracle_setup(cfg)
    th = workloads.prior_draws(4, cfg["n"], cfg["dt"], 95, logm=(5.5, 7.0))
    th[:, 14] += t0                                  # mergers inside the shifted window
    d = pipeline.aet(th[0], s)
    far = th[0].copy()
    far[8] = 1e30
    rho = np.sqrt(-2.0 * pipeline.loglike(far, s, d))
    d = d * (1000.0 / rho)
    th[0, 8] *= rho / 1000.0
    th[1] = th[0]
    th[1, 14] += 1.5                                 # a bulk walker
    lk = api.Likelihood(precision=precision, max_walkers=4, **gpu_kwargs(cfg))
    lk.set_data(_t(d))
    got = lk.loglike(_t(th)).cpu().numpy()
    for w in range(4):
        o = pipeline.loglike(th[w], s, d)
        # FP64: absolute times near 3.5e7 s carry about 500 times the rounding of the
        # one-day grids at t0 = 0 (ulp 7.5e-9 s), in the oracle and the GPU alike,
        # so the relative part of the bar scales from 1e-11 to 1e-8
        tol = max(1e-6, 1e-8 * abs(o)) if precision == 0 else max(0.05, 1e-4 * abs(o))
        assert abs(got[w] - o) <= tol, (w, got[w], o)
    lk.close()
