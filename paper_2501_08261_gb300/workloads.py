"""Seeded synthetic inputs of the paper's workload shapes.

This module holds input recipes only -- grid sizes, bands, option flags and
random parameter draws -- and none of the likelihood arithmetic.  It is the one
module that both the GPU library's tests/benchmarks and the CPU oracle's tests
use, so that both sides see identical inputs.

Shapes follow Sec. II.C / Table I of arXiv:2501.08261 (MBHB, Delta t = 5 s,
months-long signals, f_min = 1e-4 Hz, band up to 0.02 Hz).
"""
import math

import numpy as np

DAY = 86400.0

# Named workloads.  n = number of samples at dt = 5 s; orbit 0 rigid, 1 Keplerian.
CONFIGS = {
    # one day, (2,+-2) only, aligned, rigid equal arms, TDI 1.5, p = 31
    "c1_fp64_1d": dict(dt=5.0, n=17280, t0=0.0, f_lo=1e-4, f_hi=0.02, tdi_gen=15,
                       channel_mask=7, lagrange_order=31, orbit=0, mode_mask=1,
                       precessing=0),
    # sixty days, five mode pairs, aligned, Keplerian orbits, TDI 2
    "c2_hm_60d": dict(dt=5.0, n=1036800, t0=0.0, f_lo=1e-4, f_hi=0.02, tdi_gen=20,
                      channel_mask=7, lagrange_order=31, orbit=1, mode_mask=31,
                      precessing=0),
    # the same physics on shorter grids (sweep / parity sizes)
    "c2_hm_30d": dict(dt=5.0, n=518400, t0=0.0, f_lo=1e-4, f_hi=0.02, tdi_gen=20,
                      channel_mask=7, lagrange_order=31, orbit=1, mode_mask=31,
                      precessing=0),
    "c2_hm_7d": dict(dt=5.0, n=120960, t0=0.0, f_lo=1e-4, f_hi=0.02, tdi_gen=20,
                     channel_mask=7, lagrange_order=31, orbit=1, mode_mask=31,
                     precessing=0),
    "c2_hm_1d": dict(dt=5.0, n=17280, t0=0.0, f_lo=1e-4, f_hi=0.02, tdi_gen=20,
                     channel_mask=7, lagrange_order=31, orbit=1, mode_mask=31,
                     precessing=0),
    # precessing, five co-precessing modes, Keplerian, TDI 2
    "c3_prec_60d": dict(dt=5.0, n=1036800, t0=0.0, f_lo=1e-4, f_hi=0.02, tdi_gen=20,
                        channel_mask=7, lagrange_order=31, orbit=1, mode_mask=31,
                        precessing=1),
    "c3_prec_1d": dict(dt=5.0, n=17280, t0=0.0, f_lo=1e-4, f_hi=0.02, tdi_gen=20,
                       channel_mask=7, lagrange_order=31, orbit=1, mode_mask=31,
                       precessing=1),
}

DURATIONS_DAYS = (1, 7, 30, 60)                  # sweep: n = 17280, 120960, 518400, 1036800


def config(name, **override):
    c = dict(CONFIGS[name])
    c.update(override)
    return c


def _sky(rng, w):
    beta = np.arcsin(rng.uniform(-1.0, 1.0, w))
    lam = rng.uniform(0.0, 2.0 * math.pi, w)
    psi = rng.uniform(0.0, math.pi, w)
    iota = np.arccos(rng.uniform(-1.0, 1.0, w))
    phi = rng.uniform(0.0, 2.0 * math.pi, w)
    return beta, lam, psi, iota, phi


def c1_point(seed=1):
    """The single source of the one-day workload: M = 1e6 Msun, q = 2,
    chi1 = 0.5, chi2 = 0.3, merger parameter t_c = 0.75 d, sky / orientation
    drawn from ``seed``.  D = 20 Gpc (rescaled by callers to a target SNR)."""
    rng = np.random.default_rng(seed)
    beta, lam, psi, iota, phi = _sky(rng, 1)
    m1, m2 = 2.0e6 / 3.0, 1.0e6 / 3.0
    return np.array([m1, m2, 0.5, 0.0, 0.0, 0.3, 0.0, 0.0, 20.0, iota[0], phi[0],
                     beta[0], lam[0], psi[0], 0.75 * DAY])


def prior_draws(w, n, dt, seed, precessing=False, tc_frac=(0.90, 0.98),
                logm=(5.0, 7.0), q=(1.0, 8.0), logd=(0.0, 2.0)):
    """Walkers drawn from the broad priors of the throughput workloads:
    log-uniform total mass, uniform q, uniform aligned spins in [-0.99, 0.99]
    (precessing: magnitudes in [0, 0.99], isotropic tilts), isotropic sky and
    orientation, t_c uniform in a fraction of the window, D log-uniform [Gpc]."""
    rng = np.random.default_rng(seed)
    mt = 10.0 ** rng.uniform(logm[0], logm[1], w)
    qq = rng.uniform(q[0], q[1], w)
    m1 = mt * qq / (1.0 + qq)
    m2 = mt / (1.0 + qq)
    out = np.zeros((w, 15))
    out[:, 0], out[:, 1] = m1, m2
    if precessing:
        out[:, 2] = rng.uniform(0.0, 0.99, w)
        out[:, 3] = np.arccos(rng.uniform(-1.0, 1.0, w))
        out[:, 4] = rng.uniform(0.0, 2.0 * math.pi, w)
        out[:, 5] = rng.uniform(0.0, 0.99, w)
        out[:, 6] = np.arccos(rng.uniform(-1.0, 1.0, w))
        out[:, 7] = rng.uniform(0.0, 2.0 * math.pi, w)
    else:
        out[:, 2] = rng.uniform(-0.99, 0.99, w)
        out[:, 5] = rng.uniform(-0.99, 0.99, w)
    out[:, 8] = 10.0 ** rng.uniform(logd[0], logd[1], w)
    beta, lam, psi, iota, phi = _sky(rng, w)
    out[:, 9], out[:, 10], out[:, 11], out[:, 12], out[:, 13] = iota, phi, beta, lam, psi
    out[:, 14] = rng.uniform(tc_frac[0], tc_frac[1], w) * n * dt
    return out


# window lengths of the ragged workload: whole days k with k 7-smooth, so that
# n_w = 17280 k is a multiple of 64 and an FFT length of radices 2, 3, 5, 7
def _smooth(k):
    for p in (2, 3, 5, 7):
        while k % p == 0:
            k //= p
    return k == 1


RAGGED_DAYS = tuple(k for k in range(1, 61) if _smooth(k))


def newtonian_time_to_merger(m1, m2, f):
    """Newtonian (2,2) time from gravitational-wave frequency f to merger [s]."""
    mt = (m1 + m2) * 4.925490947641267e-06
    mc = mt * (m1 * m2 / (m1 + m2) ** 2) ** 0.6
    return 5.0 / 256.0 * (math.pi * f) ** (-8.0 / 3.0) * mc ** (-5.0 / 3.0)


def ragged_walkers(w, n, dt, seed, precessing=True, f_min=1e-4, pad_s=0.25 * DAY):
    """Walkers of uneven signal length on an n-sample grid: prior draws whose
    window T_w (the stretch of data up to shortly after the merger) is drawn
    log-uniformly between 1 day and the grid length, shortened to the time to
    merger from f_min plus a ringdown pad where the signal is shorter, and
    rounded to the nearest whole number of days k with k in RAGGED_DAYS; the merger
    sits at t_c = t_end - U(0.02, 0.10) T_w inside the window.  -> (params, n_w)."""
    rng = np.random.default_rng(seed + 7)
    th = prior_draws(w, n, dt, seed, precessing=precessing)
    days_max = n * dt / DAY
    nw = np.empty(w, dtype=np.int64)
    for k in range(w):
        tau = newtonian_time_to_merger(th[k, 0], th[k, 1], f_min) + pad_s
        want = days_max ** rng.uniform(0.0, 1.0)         # log-uniform in [1, days_max] d
        d = min(max(min(want, tau / DAY), 1.0), days_max)
        kd = min((q for q in RAGGED_DAYS if q <= days_max), key=lambda q: abs(q - d))
        nw[k] = int(round(kd * DAY / dt))
        th[k, 14] = n * dt - rng.uniform(0.02, 0.10) * nw[k] * dt
    return th, nw


def orbit_table_positions(t_start, dt_table, rows, seed, phase=-20.0 * math.pi / 180.0):
    """A synthetic mission orbit file: the three spacecraft's positions [m]
    at times t_start + j dt_table, shape [rows][3][3].  Each spacecraft
    follows the first-order eccentric-orbit (cartwheel) expansion about a
    1 AU circle at the sidereal rate, the constellation trailing by `phase`,
    with arms near 2.5e9 m, plus a seeded small radial breathing (1e-4 AU,
    twice a year) that makes the arms flex differently from the built-in
    models.  An input recipe: the library and the oracle resample it."""
    rng = np.random.default_rng(seed)
    au, arm = 149597870700.0, 2.5e9
    omega = 2.0 * math.pi / (365.25636 * DAY)
    e = arm / (2.0 * math.sqrt(3.0) * au)
    t = t_start + dt_table * np.arange(rows)
    a = omega * t + phase
    out = np.zeros((rows, 3, 3))
    for k in range(3):
        b = 2.0 * math.pi * k / 3.0 + phase
        x = au * np.cos(a) + au * e * (np.sin(a) * np.cos(a) * np.sin(b)
                                       - (1.0 + np.sin(a) ** 2) * np.cos(b))
        y = au * np.sin(a) + au * e * (np.sin(a) * np.cos(a) * np.cos(b)
                                       - (1.0 + np.cos(a) ** 2) * np.sin(b))
        z = -math.sqrt(3.0) * au * e * np.cos(a - b)
        breath = 1.0 + 1e-4 * np.sin(2.0 * omega * t + rng.uniform(0.0, 2.0 * math.pi))
        out[:, k, 0] = x * breath
        out[:, k, 1] = y * breath
        out[:, k, 2] = z
    return out


def table1_precessing(n, dt, tc_frac=0.9):
    """The injection of Table I (precessing columns), t_c at a fraction of the window."""
    r = math.radians
    return np.array([1.0e6, 0.7e6, 0.7, r(40.1), r(40.1), 0.4, r(22.9), r(22.9), 20.0,
                     r(149.0), r(229.2), r(-34.4), r(34.4), r(22.9), tc_frac * n * dt])


def table1_prior_box(tc, tc_halfwidth=600.0):
    """Uniform prior ranges of Table I (precessing columns, degrees -> radians),
    as (lo [15], hi [15]) in the parameter order; the merger-time range
    (t_c +- tc_halfwidth seconds) is not in Table I and is declared here."""
    r = math.radians
    lo = np.array([0.99e6, 0.69e6, 0.0, 0.0, r(-180.0), 0.0, 0.0, r(-180.0), 19.0, 0.0, 0.0,
                   r(-180.0), 0.0, r(-180.0), tc - tc_halfwidth])
    hi = np.array([1.01e6, 0.71e6, 1.0, r(180.0), r(180.0), 1.0, r(180.0), r(180.0), 21.0,
                   r(180.0), r(360.0), r(180.0), r(360.0), r(180.0), tc + tc_halfwidth])
    return lo, hi


def standard_normals(w, dim, seed):
    """Standard normal draws (used as z in theta + L z perturbations)."""
    return np.random.default_rng(seed).normal(size=(w, dim))


def _graded(nodes, g):
    """Insert nodes until adjacent spacings differ by at most a factor g either
    way: forward passes cap each spacing at g times the one before, backward
    passes at g times the one after, until a pair of passes inserts nothing."""
    def one(v):
        out = [v[0], v[1]]
        for x in v[2:]:
            while x - out[-1] > g * (out[-1] - out[-2]):
                out.append(out[-1] + max(1, int(g * (out[-1] - out[-2]))))
            out.append(x)
        return out
    cur = [int(x) for x in nodes]
    while len(cur) >= 3:
        f = one(cur)
        b = [-x for x in one([-x for x in f[::-1]])][::-1]
        if len(b) == len(cur):
            break
        cur = b
    return np.array(cur, dtype=np.int64)


def heterodyne_nodes(n, dt, m1, m2, tc, t0=0.0, df=2e-5, dt_max=43200.0, x_dense=6.0,
                     sky_pad=520.0, ring_m=200.0, f_start=1e-4, taper=1.0e4, taper_step=250.0,
                     grade=4.0):
    """Node indices of the heterodyned likelihood for a fiducial of masses m1, m2
    [Msun] and merger parameter tc [s] on an n-sample grid.

    Rule (an input choice, like the grid): a node at every sample from the
    Newtonian x = nu (tc - t) / (5 M) = x_dense through ring_m total masses
    after tc, widened by sky_pad seconds on both sides (the largest light time
    from the Sun to the constellation plus the arm); a node every taper_step
    seconds over the first `taper` seconds of the signal (from the later of t0
    and the time its Newtonian (2,2) frequency is f_start), where the start
    taper shapes the envelope; elsewhere the next node follows when the
    Newtonian (2,2) frequency has advanced by df [Hz], at least one and at most
    dt_max seconds later.  Then, where adjacent spacings differ by more than a
    factor `grade` (the dense window's end, the taper's ends), nodes are
    inserted so that the spacing changes by at most that factor: the cubic
    through four nodes then keeps a Lebesgue constant of a few, where three
    dense nodes and a 12 h one amplified the node values by up to ~1e6 across
    the long interval (grade=None keeps the raw rule).  Always holds 0 and
    n - 1."""
    mt = (m1 + m2) * 4.925490947641267e-06
    nu = m1 * m2 / (m1 + m2) ** 2
    mc = mt * nu ** 0.6
    a = tc - 5.0 * mt * x_dense / nu - sky_pad
    b = tc + ring_m * mt + sky_pad
    ia = max(0, int(math.floor((a - t0) / dt)))
    ib = min(n - 1, int(math.ceil((b - t0) / dt)))
    out = [0]
    i = 0
    while i < n - 1:
        if ia <= i < ib:
            step = 1
        else:
            tau = tc - (t0 + i * dt)
            if tau > 0.0:
                f = (5.0 / (256.0 * tau)) ** 0.375 * mc ** -0.625 / math.pi
                fdot = 96.0 / 5.0 * math.pi ** (8.0 / 3.0) * mc ** (5.0 / 3.0) * f ** (11.0 / 3.0)
                sec = min(max(df / fdot, dt), dt_max)
            else:
                sec = dt_max
            step = max(1, int(sec // dt))
            if i < ia < i + step:
                step = ia - i
        i = min(i + step, n - 1)
        out.append(i)
    ts = max(t0, tc - newtonian_time_to_merger(m1, m2, f_start))
    i0 = int(math.floor((ts - t0) / dt))
    i1 = int(math.ceil((ts + taper - t0) / dt))
    k = max(1, int(taper_step // dt))
    extra = [j for j in range(i0, i1 + 1, k) if 0 <= j < n]
    nodes = np.unique(np.array(out + extra, dtype=np.int64))
    return _graded(nodes, grade) if grade else nodes
