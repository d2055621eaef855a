"""The likelihood at the full 60-day grid (n = 1,036,800, the benchmark's
workload: five mode pairs, Keplerian orbits, TDI 2, p = 31) against the
oracle's own transform and PSD weights.

The oracle computes the data d = A,E,T of one source (zero-noise injection,
scaled to SNR 2000).  Walkers are that source at distances D' = D / s: their
A,E,T are exactly s d (the amplitude is proportional to 1/D), so the oracle's
logL = -1/2 (1 - s)^2 (d|d) follows from (d|d), which the oracle computes with
numpy's FFT.  The GPU computes every walker from its parameters through the
whole path, including the four-step FFT plan of this length and the PSD
weights of TDI 2, which no shorter parity case reaches."""
import numpy as np
import pytest

from oracle import likelihood, pipeline
from paper_2501_08261_gb300 import api, workloads

from helpers import gpu_kwargs, oracle_setup

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]
torch = pytest.importorskip("torch")

SNR = 2000.0
# s = D / D': the injection, the posterior bulk (|logL| <= ~100), further
# walkers, and h -> 0 (logL = -(d|d)/2)
SCALES = np.array([1.0, 1.0 - 2e-4, 1.0 + 3e-3, 0.995, 0.8, 0.5, 1.5, 0.0])


@pytest.fixture(scope="module")
def injection():
    from paper_2501_08261_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    cfg = workloads.config("c2_hm_60d")
    s = oracle_setup(cfg)
    th = workloads.prior_draws(1, cfg["n"], cfg["dt"], 61, logm=(5.5, 7.0))[0]
    d = pipeline.aet(th, s)
    dd = -2.0 * likelihood.loglike(np.zeros_like(d), d, s.dt, s.f_lo, s.f_hi, s.tdi_gen,
                                   s.channel_mask)
    rho = np.sqrt(dd)
    d = d * (SNR / rho)
    th = th.copy()
    th[8] *= rho / SNR
    return cfg, th, d


def _walkers(th):
    w = np.repeat(th[None], len(SCALES), axis=0)
    with np.errstate(divide="ignore"):
        w[:, 8] = np.where(SCALES > 0, th[8] / np.where(SCALES > 0, SCALES, 1.0), 1e30)
    return w


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_loglike_matches_oracle_spectrum(injection, precision):
    cfg, th, d = injection
    want = -0.5 * (1.0 - SCALES) ** 2 * SNR ** 2
    walkers = _walkers(th)
    lk = api.Likelihood(precision=precision, max_walkers=len(SCALES), **gpu_kwargs(cfg))
    lk.set_data(torch.as_tensor(d, device="cuda"))
    got = lk.loglike(torch.as_tensor(walkers, device="cuda")).cpu().numpy()
    lk.close()
    for s_, g, o in zip(SCALES, got, want):
        tol = max(1e-6, 1e-10 * abs(o)) if precision == 0 else max(0.05, 1e-4 * abs(o))
        assert abs(g - o) <= tol, (precision, s_, g, o)
