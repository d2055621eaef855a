"""Grid lengths with one prime factor in [11, 127]: the paper's 61-day window at
5 s is n = 17,280 x 61 = 2^7 3^3 5 61, whose transform needs a radix-61 stage
(fft.cu evaluates it as a direct DFT).  Parity with the oracle's numpy FFT on a
short length with the factor 61 (every walker through the whole path), and on
the 61-day grid itself by the distance-scaling argument of test_gpu_fullsize."""
import numpy as np
import pytest

from oracle import likelihood, pipeline
from paper_2501_08261_gb300 import api, workloads

from helpers import gpu_kwargs, oracle_setup

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2501_08261_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


SNR = 2000.0
SCALES = np.array([1.0, 1.0 - 2e-4, 1.0 + 3e-3, 0.8, 0.0])


def _injection(th, s):
    """(theta at distance D rho / SNR, its A,E,T) so that (d|d) = SNR^2."""
    d = pipeline.aet(th, s)
    dd = -2.0 * likelihood.loglike(np.zeros_like(d), d, s.dt, s.f_lo, s.f_hi, s.tdi_gen,
                                   s.channel_mask)
    rho = np.sqrt(dd)
    th = th.copy()
    th[8] *= rho / SNR
    return th, d * (SNR / rho)


@pytest.mark.parametrize("precision", [0, 1])
def test_length_with_factor_61_matches_oracle(precision):
    cfg = workloads.config("c2_hm_1d", n=61 * 320)
    s = oracle_setup(cfg)
    th = workloads.prior_draws(3, cfg["n"], cfg["dt"], 17, logm=(5.5, 7.0))
    th[0], d = _injection(th[0], s)      # SNR 2000, as in the other mixed parity tests
    want = np.array([pipeline.loglike(t, s, d) for t in th])
    lk = api.Likelihood(precision=precision, max_walkers=3, **gpu_kwargs(cfg))
    lk.set_data(torch.as_tensor(d, device="cuda"))
    got = lk.loglike(torch.as_tensor(th, device="cuda")).cpu().numpy()
    lk.close()
    for g, o in zip(got, want):
        tol = max(1e-6, 1e-10 * abs(o)) if precision == 0 else max(0.05, 1e-4 * abs(o))
        assert abs(g - o) <= tol, (precision, g, o)


@pytest.fixture(scope="module")
def sixty_one_days():
    cfg = workloads.config("c2_hm_60d", n=17280 * 61)
    s = oracle_setup(cfg)
    th = workloads.prior_draws(1, cfg["n"], cfg["dt"], 61, logm=(5.5, 7.0))[0]
    return (cfg,) + _injection(th, s)


@pytest.mark.parametrize("precision", [0, 1])
def test_sixty_one_day_window_matches_oracle_spectrum(sixty_one_days, precision):
    """n = 1,054,080: walkers are the injection at distances D / s, whose A, E, T
    are s d exactly, so the oracle's logL = -1/2 (1 - s)^2 (d|d)."""
    cfg, th, d = sixty_one_days
    w = np.repeat(th[None], len(SCALES), axis=0)
    w[:, 8] = np.where(SCALES > 0, th[8] / np.where(SCALES > 0, SCALES, 1.0), 1e30)
    want = -0.5 * (1.0 - SCALES) ** 2 * SNR ** 2
    lk = api.Likelihood(precision=precision, max_walkers=len(SCALES), **gpu_kwargs(cfg))
    lk.set_data(torch.as_tensor(d, device="cuda"))
    got = lk.loglike(torch.as_tensor(w, device="cuda")).cpu().numpy()
    lk.close()
    for s_, g, o in zip(SCALES, got, want):
        tol = max(1e-6, 1e-10 * abs(o)) if precision == 0 else max(0.05, 1e-4 * abs(o))
        assert abs(g - o) <= tol, (precision, s_, g, o)
