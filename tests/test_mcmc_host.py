"""Host-side chain analysis of paper_2501_08261_gb300.mcmc: the integrated
autocorrelation time against the closed form of an AR(1) process."""
import numpy as np

from paper_2501_08261_gb300 import mcmc


def test_integrated_time_of_ar1_matches_closed_form():
    # x_t = r x_{t-1} + e_t has tau = (1 + r) / (1 - r)
    rng = np.random.default_rng(0)
    N, W = 20000, 32
    for r in (0.0, 0.5, 0.9):
        x = np.zeros((N, W))
        e = rng.normal(size=(N, W))
        for t in range(1, N):
            x[t] = r * x[t - 1] + e[t]
        tau = mcmc.integrated_time(x)
        want = (1 + r) / (1 - r)
        assert abs(tau - want) <= 0.08 * want, (r, tau, want)


def test_frozen_chain_has_no_effective_samples_beyond_one_per_walker():
    chain = np.zeros((100, 4, 15))
    n, tau = mcmc.ess(chain, [0, 1])
    assert tau == 100.0 and n == 4.0
