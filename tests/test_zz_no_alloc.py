"""lisa_td_residual_loglike_noalloc: the DFT + PSD-weighted norm for callers
that must not allocate device memory (their memory sits in a framework's
caching pool, or their loop cannot take the synchronisation cudaFree implies).
Its scratch is a fixed static device array, so it must give what
lisa_td_loglike_batch gives for the same walkers, call after call, and refuse
sizes the array cannot hold.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2501_08261_gb300 import api, workloads

from helpers import gpu_kwargs

torch = pytest.importorskip("torch")


def test_rejects_sizes_beyond_the_static_scratch():
    # the size and shape checks return before any CUDA call, so no GPU is needed
    lib = api.load_library(api._build.build())
    fake = ctypes.c_void_p(1 << 20)                   # never dereferenced
    big = api.make_config(dt=5.0, n=1036800, precision=0)
    assert lib.lisa_td_residual_loglike_noalloc(ctypes.byref(big), fake, 2, fake, None) == -5
    assert b"scratch" in lib.lisa_td_last_error()
    ok = api.make_config(dt=5.0, n=17280, precision=0)
    assert lib.lisa_td_residual_loglike_noalloc(ctypes.byref(ok), fake, 80, fake, None) == -5
    assert lib.lisa_td_residual_loglike_noalloc(ctypes.byref(ok), fake, 3, fake, None) == -1
    assert b"even" in lib.lisa_td_last_error()
    assert lib.lisa_td_residual_loglike_noalloc(ctypes.byref(ok), None, 2, fake, None) == -1
    inf_dt = api.make_config(dt=float("inf"), n=17280, precision=1)
    assert lib.lisa_td_residual_loglike_noalloc(ctypes.byref(inf_dt), fake, 2, fake, None) == -1
    assert b"dt" in lib.lisa_td_last_error()
    # the mixed path's boundary at n = 17280: W = 158 needs more than the array
    mixed = api.make_config(dt=5.0, n=17280, precision=1)
    assert lib.lisa_td_residual_loglike_noalloc(ctypes.byref(mixed), fake, 158, fake, None) == -5
    if not torch.cuda.is_available():
        # W = 156 (and W = 78 in FP64) pass every size check and stop only at the
        # first CUDA call, which fails on a machine without a GPU; on a GPU
        # machine the fake pointers would be used, so this part runs only here
        assert lib.lisa_td_residual_loglike_noalloc(ctypes.byref(mixed), fake, 156, fake, None) == -3
        assert lib.lisa_td_residual_loglike_noalloc(ctypes.byref(ok), fake, 78, fake, None) == -3


def test_grid_length_rule():
    """FFT lengths: 2^a 3^b 5^c 7^d times at most one prime in [11, 127].  The
    plan is checked before any CUDA call, so no GPU is needed for the refusals."""
    lib = api.load_library(api._build.build())
    fake = ctypes.c_void_p(1 << 20)                   # never dereferenced
    for n in (64 * 11 * 13, 64 * 131, 64 * 61 * 61, 17280 * 11 * 11):
        cfg = api.make_config(dt=5.0, n=n, precision=1)
        assert lib.lisa_td_residual_loglike_noalloc(ctypes.byref(cfg), fake, 2, fake, None) == -1, n
        assert b"prime" in lib.lisa_td_last_error() or b"2^" in lib.lisa_td_last_error(), n
    if not torch.cuda.is_available():
        # accepted lengths pass the plan and stop at the first CUDA call
        for n in (64 * 61, 64 * 11, 64 * 127, 2 ** 6 * 3 ** 3 * 5 * 61):
            cfg = api.make_config(dt=5.0, n=n, precision=1)
            assert lib.lisa_td_residual_loglike_noalloc(ctypes.byref(cfg), fake, 2, fake, None) == -3, n


def _walkers(cfg, w, seed):
    return workloads.prior_draws(w, cfg["n"], cfg["dt"], seed, logm=(5.5, 7.0))


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.gpu
@pytest.mark.parametrize("name,precision", [("c1_fp64_1d", 0), ("c2_hm_1d", 1)])
def test_noalloc_matches_loglike_batch_on_two_calls(name, precision):
    from paper_2501_08261_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    cfg = workloads.config(name)
    kw = gpu_kwargs(cfg)
    ref = api.Likelihood(precision=0, max_walkers=8, **kw)
    lk = api.Likelihood(precision=precision, max_walkers=8, **kw)
    truth = _walkers(cfg, 1, 71)
    d = ref.tdi(ref.project(_t(truth)))[:, :, 0].contiguous()     # zero-noise injection
    lk.set_data(d)
    if precision == 0:
        def close(g, o):
            return abs(g - o) <= max(1e-6, 1e-11 * abs(o))     # the FP64 tests' bar
    else:
        def close(g, o):
            return abs(g - o) <= max(0.05, 1e-4 * abs(o))      # the mixed tests' bar
    for call, (W, seed) in enumerate(((6, 72), (4, 73))):    # two calls in a row
        th = _walkers(cfg, W, seed)
        th[0] = truth[0]
        want = lk.loglike(_t(th)).cpu().numpy()
        r = (lk.tdi(lk.project(_t(th))) - d.to(lk.dtype)[:, :, None]).contiguous()
        got = torch.full((W,), float("nan"), dtype=torch.float64, device="cuda")
        api.lisa_td_residual_loglike_noalloc(lk.cfg, r, W, got)
        got = got.cpu().numpy()
        assert np.all(np.isfinite(got)), (call, got)
        for w in range(W):
            assert close(got[w], want[w]), (call, w, got[w], want[w])
    lk.close()
    ref.close()


@pytest.mark.gpu
@pytest.mark.parametrize("n", [3136, 20160, 21952])     # 2^6 7^2, 2^6 3^2 5 7, 2^6 7^3
@pytest.mark.parametrize("precision", [0, 1])
def test_residual_norm_at_radix7_lengths_matches_oracle(n, precision):
    """The DFT + PSD-weighted norm alone (Sec. II.B inner product) at lengths
    whose FFT plans use radix-7 (and 5, 3) stages, against the oracle's
    likelihood on the same residual.  The mixed path gets the oracle's
    residual rounded to FP32, so only its FFT and norm arithmetic is compared:
    a relative bar of 2e-5 on a sum of ~n/10 positive terms."""
    _norm_case(n, precision)


@pytest.mark.gpu
@pytest.mark.parametrize("n", [3904, 8128, 2112, 40640])
@pytest.mark.parametrize("precision", [0, 1])
def test_residual_norm_at_prime_factor_lengths_matches_oracle(n, precision):
    """As above, at lengths with one prime factor in [11, 127], whose plans
    end a pass with the direct prime-radix stage: n1 = 61 (odd, the stage
    alone), n2 = 127, n1 = 44 = 4 x 11 and n2 = 254 = 2 x 127 (the stage
    after others, with its twiddle sweep)."""
    _norm_case(n, precision)


def _norm_case(n, precision):
    from oracle import likelihood
    from paper_2501_08261_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    W = 4
    rng = np.random.default_rng(n + 10 * precision)
    r = rng.normal(size=(3, n, W)) * 1e-21
    if precision == 1:
        r = r.astype(np.float32).astype(np.float64)
    cfg = api.make_config(dt=5.0, n=n, precision=precision, tdi_gen=20)
    rt = torch.as_tensor(r, dtype=torch.float64 if precision == 0 else torch.float32,
                         device="cuda").contiguous()
    got = torch.full((W,), float("nan"), dtype=torch.float64, device="cuda")
    api.lisa_td_residual_loglike_noalloc(cfg, rt, W, got)
    got = got.cpu().numpy()
    zero = np.zeros((3, n))
    for w in range(W):
        want = likelihood.loglike(r[:, :, w], zero, 5.0, cfg.f_lo, cfg.f_hi, 20, 7)
        bar = 1e-11 * abs(want) if precision == 0 else 2e-5 * abs(want)
        assert abs(got[w] - want) <= bar, (n, precision, w, got[w], want)
