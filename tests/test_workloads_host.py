"""Host-side checks of the seeded input generators (no GPU): the ragged
windows are whole 7-smooth days that tile evenly, each walker's merger sits
inside its window, the draws are reproducible from their seeds and stay in
their stated ranges, and the Table I injection lies inside the Table I box."""
import math

import numpy as np
import pytest

from paper_2501_08261_gb300 import workloads

DT = 5.0
SAMPLES_PER_DAY = int(workloads.DAY / DT)       # 17280


def _factor_7smooth(k):
    for p in (2, 3, 5, 7):
        while k % p == 0:
            k //= p
    return k == 1


def test_ragged_days_are_the_7_smooth_whole_days():
    assert workloads.RAGGED_DAYS == tuple(k for k in range(1, 61) if _factor_7smooth(k))
    assert workloads.RAGGED_DAYS[:8] == (1, 2, 3, 4, 5, 6, 7, 8)
    assert 11 not in workloads.RAGGED_DAYS and 60 in workloads.RAGGED_DAYS
    for k in workloads.RAGGED_DAYS:
        n = k * SAMPLES_PER_DAY
        assert n % 64 == 0                       # whole TDI tiles
        assert _factor_7smooth(n)                # an FFT length of radices 2, 3, 5, 7


@pytest.mark.parametrize("seed", [4, 9])
def test_ragged_walkers_windows_and_merger_times(seed):
    n = 60 * SAMPLES_PER_DAY
    th, nw = workloads.ragged_walkers(256, n, DT, seed)
    th2, nw2 = workloads.ragged_walkers(256, n, DT, seed)
    assert np.array_equal(th, th2) and np.array_equal(nw, nw2)      # seeded
    days = nw // SAMPLES_PER_DAY
    assert np.all(nw == days * SAMPLES_PER_DAY)
    assert set(days.tolist()) <= set(workloads.RAGGED_DAYS)
    assert days.min() >= 1 and days.max() <= 60
    assert len(np.unique(days)) > 5                                  # uneven durations
    # merger inside the walker's own (end-aligned) window, 2-10 % before its end
    before_end = n * DT - th[:, 14]
    assert np.all(before_end >= 0.02 * nw * DT - 1e-6)
    assert np.all(before_end <= 0.10 * nw * DT + 1e-6)
    # windows spread over the whole 1-60 d span (log-uniform draws)
    assert days.min() <= 2 and days.max() >= 30
    # a window is never much longer than the signal it holds: at most the time
    # to merger from f_min plus the pad, rounded to the nearest 7-smooth day
    smooth = np.array(workloads.RAGGED_DAYS)
    for k in range(256):
        tau = workloads.newtonian_time_to_merger(th[k, 0], th[k, 1], 1e-4) + 0.25 * workloads.DAY
        cap = min(max(tau / workloads.DAY, 1.0), 60.0)
        nearest = smooth[np.argmin(np.abs(smooth - cap))]
        assert days[k] <= max(nearest, cap) + 1e-9, (k, days[k], cap)


def test_newtonian_time_to_merger_scalings():
    # tau ~ f^(-8/3) M_c^(-5/3): the chirp mass fixes it (equal chirp mass, equal tau)
    t0 = workloads.newtonian_time_to_merger(1e6, 1e6, 1e-4)
    assert workloads.newtonian_time_to_merger(1e6, 1e6, 2e-4) == pytest.approx(t0 * 2 ** (-8 / 3))
    assert workloads.newtonian_time_to_merger(2e6, 2e6, 1e-4) == pytest.approx(t0 * 2 ** (-5 / 3))
    # chirp mass of (m1, m2) = (3, 1) x 1e6 equals that of an equal-mass pair of m each, with
    # m = M_c 2^(1/5): the times agree
    mc = (3e6 * 1e6) ** 0.6 / (4e6) ** 0.2
    m = mc * 2 ** 0.2
    assert workloads.newtonian_time_to_merger(3e6, 1e6, 1e-4) == pytest.approx(
        workloads.newtonian_time_to_merger(m, m, 1e-4), rel=1e-12)


@pytest.mark.parametrize("precessing", [False, True])
def test_prior_draws_ranges_and_seeds(precessing):
    n = SAMPLES_PER_DAY
    th = workloads.prior_draws(500, n, DT, 3, precessing=precessing)
    assert np.array_equal(th, workloads.prior_draws(500, n, DT, 3, precessing=precessing))
    assert not np.array_equal(th, workloads.prior_draws(500, n, DT, 4, precessing=precessing))
    mt = th[:, 0] + th[:, 1]
    assert np.all((mt >= 1e5 * (1 - 1e-12)) & (mt <= 1e7 * (1 + 1e-12)))
    q = th[:, 0] / th[:, 1]
    assert np.all((q >= 1 - 1e-12) & (q <= 8 + 1e-12))
    if precessing:
        assert np.all((th[:, 2] >= 0) & (th[:, 2] <= 0.99) & (th[:, 5] >= 0) & (th[:, 5] <= 0.99))
        assert np.all((th[:, 3] >= 0) & (th[:, 3] <= math.pi))
    else:
        assert np.all(np.abs(th[:, [2, 5]]) <= 0.99)
        assert np.all(th[:, [3, 4, 6, 7]] == 0.0)
    assert np.all((th[:, 8] >= 1.0) & (th[:, 8] <= 100.0))
    assert np.all(np.abs(th[:, 11]) <= math.pi / 2)                     # ecliptic latitude
    assert np.all((th[:, 14] >= 0.90 * n * DT) & (th[:, 14] <= 0.98 * n * DT))


def test_table1_injection_lies_inside_the_table1_box():
    n = SAMPLES_PER_DAY
    inj = workloads.table1_precessing(n, DT)
    lo, hi = workloads.table1_prior_box(inj[14])
    assert np.all(lo < inj) and np.all(inj < hi)
    assert inj[0] >= inj[1]                                             # m1 >= m2


def test_named_configs_sizes():
    c = workloads.config("c2_hm_60d")
    assert c["n"] == 60 * SAMPLES_PER_DAY and c["dt"] == DT
    assert (c["tdi_gen"], c["orbit"], c["mode_mask"], c["lagrange_order"]) == (20, 1, 31, 31)
    assert workloads.config("c2_hm_60d", n=4320)["n"] == 4320          # overrides
    for name in ("c1_fp64_1d", "c2_hm_1d", "c3_prec_1d"):
        assert workloads.config(name)["n"] == SAMPLES_PER_DAY
