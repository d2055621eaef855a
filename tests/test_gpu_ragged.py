"""Ragged batches (lisa_td_loglike_ragged): each walker on its own window of
the last n_w samples equals the plain likelihood on a context whose grid is
that window (and the oracle on it), with and without CUDA-graph replay."""
import numpy as np
import pytest

from oracle import pipeline
from paper_2501_08261_gb300 import api, workloads

from helpers import gpu_kwargs, oracle_setup

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]
torch = pytest.importorskip("torch")
DAY = 17280


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2501_08261_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _walkers(n, windows, seed, precessing):
    rng = np.random.default_rng(seed)
    W = len(windows)
    th = workloads.prior_draws(W, n, 5.0, seed, precessing=precessing, logm=(5.5, 6.5))
    th[:, 14] = n * 5.0 - rng.uniform(0.05, 0.3, W) * np.asarray(windows) * 5.0
    return th


def _bar(want, dd, precision):
    """|dlogL| bar between two evaluations of the same window.  logL =
    -1/2 (r|r) with r = h - d, so a norm-relative error eps on the series moves
    logL by up to eps ||r|| ||d|| = eps sqrt(2|logL| 2|logL_0|) (logL_0 =
    -1/2 (d|d)); eps = 1e-10 for FP64 (the series tolerance of the FP64 tests),
    2e-6 for two mixed evaluations on different tilings (each within ~2e-6
    relative of FP64 on loud walkers, 50x inside the mixed path's far-walker
    bar of 1e-4); and never below the fixed floors."""
    eps, floor, rel = (1e-10, 1e-6, 1e-10) if precision == 0 else (2e-6, 1e-3, 2e-6)
    return max(floor, rel * abs(want), eps * np.sqrt(4.0 * abs(want) * abs(dd)))


def _window_ctx(cfg, nw, precision, W, d):
    kw = gpu_kwargs(cfg)
    kw["n"] = nw
    kw["t0"] = cfg["t0"] + (cfg["n"] - nw) * cfg["dt"]
    lk = api.Likelihood(precision=precision, max_walkers=W, **kw)
    lk.set_data(d[:, cfg["n"] - nw:].contiguous())
    return lk


@pytest.mark.parametrize("name,precision", [("c2_hm_1d", 0), ("c3_prec_1d", 0), ("c2_hm_1d", 1),
                                            ("c3_prec_1d", 1)])
def test_ragged_equals_per_window_likelihood(name, precision):
    cfg = workloads.config(name, n=4 * DAY)
    windows = np.array([2, 4, 1, 4, 2, 1, 4, 3, 2]) * DAY          # classes 1, 2, 3, 4 days
    th = _walkers(cfg["n"], windows, 11, bool(cfg["precessing"]))
    ref = api.Likelihood(precision=0, max_walkers=len(th), **gpu_kwargs(cfg))
    d = ref.tdi(ref.project(_t(th[:1])))[:, :, 0].contiguous()
    lk = api.Likelihood(precision=precision, max_walkers=len(th), **gpu_kwargs(cfg))
    lk.set_data(d)
    got, st = lk.loglike_ragged(_t(th), windows, with_status=True)
    got = got.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    for nw in np.unique(windows):
        sel = np.nonzero(windows == nw)[0]
        wl = _window_ctx(cfg, int(nw), precision, len(sel), d)
        want = wl.loglike(_t(th[sel])).cpu().numpy()
        far = th[sel].copy()
        far[:, 8] = 1e30                                        # h -> 0: -1/2 (d|d)
        dd = wl.loglike(_t(far)).cpu().numpy()
        for k, w in enumerate(sel):
            assert abs(got[w] - want[k]) <= _bar(want[k], dd[k], precision), (nw, w, got[w], want[k])
        wl.close()
    lk.close()
    ref.close()


def test_ragged_matches_oracle():
    cfg = workloads.config("c2_hm_1d", n=2 * DAY)
    windows = np.array([2 * DAY, DAY, 2 * DAY])
    th = _walkers(cfg["n"], windows, 12, False)
    s = oracle_setup(cfg)
    d = pipeline.aet(th[0], s)
    lk = api.Likelihood(precision=0, max_walkers=3, **gpu_kwargs(cfg))
    lk.set_data(_t(d))
    got = lk.loglike_ragged(_t(th), windows).cpu().numpy()
    for w in range(3):
        off = cfg["n"] - windows[w]
        sw = oracle_setup(dict(cfg, n=int(windows[w]), t0=cfg["t0"] + off * cfg["dt"]))
        want = pipeline.loglike(th[w], sw, d[:, off:])
        far = th[w].copy()
        far[8] = 1e30
        dd = pipeline.loglike(far, sw, d[:, off:])
        assert abs(got[w] - want) <= _bar(want, dd, 0), (w, got[w], want)
    lk.close()


def test_graph_replay_and_recapture_and_errors():
    cfg = workloads.config("c2_hm_1d", n=4 * DAY)
    windows = np.array([DAY, 2 * DAY, 4 * DAY, DAY, 2 * DAY, 4 * DAY])
    th = _walkers(cfg["n"], windows, 13, False)
    lk = api.Likelihood(precision=1, max_walkers=8, **gpu_kwargs(cfg))
    ref = api.Likelihood(precision=0, max_walkers=8, **gpu_kwargs(cfg))
    d = ref.tdi(ref.project(_t(th[:1])))[:, :, 0].contiguous()
    lk.set_data(d)
    plain = lk.loglike_ragged(_t(th), windows).cpu().numpy()
    api.lisa_td_ragged_graph(lk.ctx, 1)
    stream = torch.cuda.Stream()
    params = _t(th)
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(3):                                   # capture, then replays
            out.fill_(0.0)
            api.lisa_td_loglike_ragged(lk.ctx, params, 6, windows, out, None, stream)
    stream.synchronize()
    assert np.array_equal(out.cpu().numpy(), plain)
    w2 = windows.copy()
    w2[0] = 3 * DAY                                          # new histogram: recapture
    with torch.cuda.stream(stream):
        api.lisa_td_loglike_ragged(lk.ctx, params, 6, w2, out, None, stream)
    stream.synchronize()
    api.lisa_td_ragged_graph(lk.ctx, 0)
    again = lk.loglike_ragged(_t(th), w2).cpu().numpy()
    assert np.array_equal(out.cpu().numpy(), again)
    # the other walkers keep their windows (a different pairing inside the FFT
    # changes only rounding)
    assert again[0] != plain[0]
    assert np.all(np.abs(again[1:] - plain[1:]) <= np.maximum(1e-3, 1e-6 * np.abs(plain[1:])))
    for bad in (DAY + 1, 5 * DAY, 64):
        wb = windows.copy()
        wb[2] = bad
        with pytest.raises(api.LisaTdError):
            lk.loglike_ragged(_t(th), wb)
    lk.close()
    ref.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_tiled_and_per_class_paths_agree(precision):
    """32 walkers in three odd-sized classes: a context with room for the
    padding columns runs the tiled path, one without falls back to per-class
    launches; both give the per-window likelihood."""
    cfg = workloads.config("c3_prec_1d", n=4 * DAY)
    windows = np.array([4] * 11 + [2] * 11 + [1] * 10) * DAY
    np.random.default_rng(3).shuffle(windows)
    th = _walkers(cfg["n"], windows, 14, True)
    ref = api.Likelihood(precision=0, max_walkers=32, **gpu_kwargs(cfg))
    d = ref.tdi(ref.project(_t(th[:1])))[:, :, 0].contiguous()
    tiled = api.Likelihood(precision=precision, max_walkers=64, **gpu_kwargs(cfg))
    per_class = api.Likelihood(precision=precision, max_walkers=32, **gpu_kwargs(cfg))
    tiled.set_data(d)
    per_class.set_data(d)
    a = tiled.loglike_ragged(_t(th), windows).cpu().numpy()
    b = per_class.loglike_ragged(_t(th), windows).cpu().numpy()
    far = th.copy()
    far[:, 8] = 1e30
    dd = per_class.loglike_ragged(_t(far), windows).cpu().numpy()
    for w in range(len(th)):
        assert abs(a[w] - b[w]) <= _bar(b[w], dd[w], precision), (w, a[w], b[w])
    for lk in (ref, tiled, per_class):
        lk.close()
