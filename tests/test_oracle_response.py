"""Pins of the oracle's response stage (Sec. II.B) against closed forms,
invariants and special cases -- none of them re-types the oracle's formulas."""
import math

import numpy as np
import pytest

from oracle import consts as K
from oracle import orbits, response

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# --------------------------------------------------------------- Lagrange ---
@pytest.mark.parametrize("p", [1, 7, 15, 31])
def test_lagrange_exact_on_polynomials(p):
    rng = np.random.default_rng(p)
    n = 200
    c = rng.normal(size=p + 1)
    poly = lambda x: np.polynomial.polynomial.polyval((x - 100.0) / 16.0, c)
    series = poly(np.arange(n, dtype=np.float64))
    tau = 100.0 + rng.uniform(-0.5, 1.0, size=64)
    got = response.interp(series, tau, p)
    want = poly(tau)
    assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(series[84:118]))


def test_lagrange_degree_p_plus_one_is_not_exact():
    # a plausible mistake (one node short) would still pass the test above for
    # lower degrees; degree p+1 must show an interpolation error
    p = 7
    x = np.arange(100, dtype=np.float64)
    series = ((x - 50.0) / 4.0) ** (p + 1)
    got = response.interp(series, np.array([50.37]), p)
    assert abs(got[0] - ((0.37) / 4.0) ** (p + 1)) > 1e-6


def test_lagrange_linear_and_integer_positions():
    rng = np.random.default_rng(0)
    s = rng.normal(size=50)
    tau = np.array([3.25, 10.5, 20.75])
    lin = s[[3, 10, 20]] * (1 - (tau % 1)) + s[[4, 11, 21]] * (tau % 1)
    assert np.allclose(response.interp(s, tau, 1), lin, rtol=0, atol=1e-15)
    for p in (1, 31):
        assert np.allclose(response.interp(s, np.arange(16, 30.0), p), s[16:30],
                           rtol=0, atol=1e-13)


def test_lagrange_zero_outside_grid():
    s = np.ones(40)
    # far outside: every node is off the grid
    assert response.interp(s, np.array([-100.3, 200.7]), 31).tolist() == [0.0, 0.0]


# ------------------------------------------------------------ TDI tables ---
def test_x2_table_is_x15_minus_x15_delayed_by_round_trip():
    """Every X_2 term is an X_1.5 term, or an X_1.5 term delayed by
    R = L2 + L-2 + L3 + L-3 with its sign flipped (the reading of the
    y_123 delay typo restores this structure)."""
    R = (2, -2, 3, -3)
    expect = {(l, s, tuple(sorted(d))) for (l, s, d) in response.X15_TERMS}
    expect |= {(l, -s, tuple(sorted(d + R))) for (l, s, d) in response.X15_TERMS}
    got = {(l, s, tuple(sorted(d))) for (l, s, d) in response.X20_TERMS}
    assert got == expect and len(response.X20_TERMS) == 16


def test_cyclic_permutation_of_links():
    assert [response.cyclic(l) for l in (1, 2, 3, -1, -2, -3)] == [2, 3, 1, -2, -3, -1]
    for l in orbits.LINKS:
        s, r = orbits.LINK_ENDS[l]
        s2, r2 = orbits.LINK_ENDS[response.cyclic(l)]
        assert (s2, r2) == (s % 3 + 1, r % 3 + 1)


def test_link_ends_match_printed_labels():
    # y_{1-32}: s=1, l=-3, r=2 ; y_{231}: s=2,l=3,r=1 ; y_{123} ; y_{3-21}
    assert orbits.LINK_ENDS[-3] == (1, 2)
    assert orbits.LINK_ENDS[3] == (2, 1)
    assert orbits.LINK_ENDS[2] == (1, 3)
    assert orbits.LINK_ENDS[-2] == (3, 1)
    for l in (1, 2, 3):              # link |l| joins the two craft other than |l|
        assert set(orbits.LINK_ENDS[l]) == {1, 2, 3} - {l}
        assert orbits.LINK_ENDS[-l] == orbits.LINK_ENDS[l][::-1]


# ------------------------------------------------------- zero waveform -----
def test_zero_waveform_gives_zero_tdi():
    n = 600
    z = np.zeros(n)
    y = response.all_links(z, z, 0.0, 5.0, "kepler", 0.3, 1.1, 31)
    assert all(np.all(v == 0.0) for v in y.values())
    X, Y, Z = response.tdi_xyz(y, n, 0.0, 5.0, "kepler", 20, 31)
    A, E, T = response.aet_from_xyz(X, Y, Z)
    assert np.all(A == 0) and np.all(E == 0) and np.all(T == 0)


# -------------------------- static constellation, monochromatic plane wave --
def _analytic_y(link, t, w, amp, orbit, beta, lam):
    """Exact y for h+ = amp cos(w t), hx = 0 (no interpolation)."""
    k, u, v = response.source_basis(beta, lam)
    rr, rs, n, L = orbits.link_geometry(orbit, link, t)
    ts = t - L - rs @ k
    tr = t - rr @ k
    un, vn = n @ u, n @ v
    return (un * un - vn * vn) * amp * (np.cos(w * ts) - np.cos(w * tr)) / (2 * (1 - n @ k))


@pytest.mark.parametrize("gen", [15, 20])
@pytest.mark.parametrize("orbit", ["static_rigid", "static_kepler"])
def test_static_monochromatic_tdi_matches_closed_form(gen, orbit):
    dt, n = 5.0, 1200
    f = 0.0123
    w, amp = 2 * math.pi * f, 1e-21
    beta, lam = -0.6, 0.6
    t = np.arange(n) * dt
    hp, hc = amp * np.cos(w * t), np.zeros(n)
    y = response.all_links(hp, hc, 0.0, dt, orbit, beta, lam, 31)
    idx = np.arange(300, 900)
    X, Y, Z = response.tdi_xyz(y, n, 0.0, dt, orbit, gen, 31, idx)
    tt = idx * dt
    want = []
    for ch in range(3):
        acc = np.zeros(idx.shape)
        for (link, sg, dl) in response.channel_terms(gen, ch):
            D = sum((orbits.light_time(orbit, d, tt) for d in dl), np.zeros(idx.shape))
            acc += sg * _analytic_y(link, tt - D, w, amp, orbit, beta, lam)
        want.append(acc)
    for got, ref in zip((X, Y, Z), want):
        assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_static_equal_arm_transfer_function():
    """Static equal arms, X_1.5 of a monochromatic wave has the textbook
    transfer |X| ~ 2 sin(w L) * |y-combination| -> zeros at f = k/(2L)."""
    dt, n, orbit = 1.0, 1200, "static_rigid"
    f = 1.0 / (2 * K.ARM_S)                   # sin(2 pi f L) = 0: X_1.5 vanishes
    w, amp = 2 * math.pi * f, 1e-21
    t = np.arange(n) * dt
    y = response.all_links(amp * np.cos(w * t), np.zeros(n), 0.0, dt, orbit, 0.2, 2.0, 31)
    yscale = max(np.max(np.abs(v[300:900])) for v in y.values())
    X, Y, Z = response.tdi_xyz(y, n, 0.0, dt, orbit, 15, 31, np.arange(300, 900))
    assert np.max(np.abs(X)) < 1e-8 * yscale


# ------------------------------------------------- laser-noise cancellation -
def _laser(k, t):
    rng = np.random.default_rng(100 + k)
    fr = rng.uniform(0.001, 0.02, 8)
    ph = rng.uniform(0, 2 * math.pi, 8)
    return np.sum(np.cos(2 * math.pi * fr[:, None] * t[None, :] + ph[:, None]), axis=0)


def _laser_links(orbit, n, dt):
    t = np.arange(n) * dt
    y = {}
    for l in orbits.LINKS:
        s, r = orbits.LINK_ENDS[l]
        L = orbits.light_time(orbit, l, t)
        y[l] = _laser(s, t - L) - _laser(r, t)
    return y


@pytest.mark.parametrize("gen", [15, 20])
def test_laser_noise_cancels_static_unequal_arms(gen):
    orbit, n, dt = "static_kepler", 2000, 1.0
    y = _laser_links(orbit, n, dt)
    scale = np.max(np.abs(y[1]))
    X, Y, Z = response.tdi_xyz(y, n, 0.0, dt, orbit, gen, 31, np.arange(400, 1600))
    for c in (X, Y, Z):
        assert np.max(np.abs(c)) < 1e-9 * scale


def test_printed_x2_typo_leaves_laser_noise():
    """With the y_123 delay exactly as printed the two terms do not cancel the
    laser noise, which is why the reading above is taken."""
    orbit, n, dt = "static_kepler", 2000, 1.0
    y = _laser_links(orbit, n, dt)
    printed = list(response.X20_TERMS)
    printed[10] = (2, +1, (-2, -2, 2, 3, -3))
    t = np.arange(400, 1600) * dt
    L = {l: orbits.light_time(orbit, l, t) for l in orbits.LINKS}
    X = np.zeros(t.shape)
    for (link, sg, dl) in printed:
        D = sum((L[d] for d in dl), np.zeros(t.shape))
        X += sg * response.interp(y[link], t / dt - D / dt, 31)
    assert np.max(np.abs(X)) > 1e-3 * np.max(np.abs(y[1]))


def test_equal_arms_x2_is_x15_minus_delayed_x15():
    orbit, n, dt = "rigid", 3000, 5.0
    rng = np.random.default_rng(7)
    y = {l: np.convolve(rng.normal(size=n), np.hanning(40), mode="same") for l in orbits.LINKS}
    idx = np.arange(600, 2400)
    X2 = response.tdi_xyz(y, n, 0.0, dt, orbit, 20, 31, idx)[0]
    X15 = response.tdi_xyz(y, n, 0.0, dt, orbit, 15, 31, idx)[0]
    # X_1.5 at t - 4L: every X_1.5 delay lengthened by 4L
    X15d = np.zeros(idx.shape)
    for (link, sg, dl) in response.X15_TERMS:
        D = (len(dl) + 4) * K.ARM_S
        X15d += sg * response.interp(y[link], idx - D / dt, 31)
    assert np.max(np.abs(X2 - (X15 - X15d))) < 1e-12 * np.max(np.abs(X15))


# -------------------------------------------------- polarisation frame -----
def test_y_invariant_under_joint_rotation_of_polarisation_frame():
    """Rotating (u, v) by delta and (h+, hx) by -2 delta leaves y unchanged only
    with the cross term 2 x_x (the n_i n_j h_ij / 2 reading of Eq. yslr)."""
    rng = np.random.default_rng(3)
    n, dt, beta, lam, p = 800, 5.0, 0.4, 2.5, 31
    hp = np.convolve(rng.normal(size=n), np.hanning(30), mode="same")
    hc = np.convolve(rng.normal(size=n), np.hanning(30), mode="same")
    delta = 0.37
    k, u, v = response.source_basis(beta, lam)
    u2 = math.cos(delta) * u + math.sin(delta) * v
    v2 = -math.sin(delta) * u + math.cos(delta) * v
    hp2 = math.cos(2 * delta) * hp + math.sin(2 * delta) * hc
    hc2 = -math.sin(2 * delta) * hp + math.cos(2 * delta) * hc
    idx = np.arange(200, 600)
    t = idx * dt
    for link in orbits.LINKS:
        rr, rs, nn, L = orbits.link_geometry("kepler", link, t)
        ts, tr = t - L - rs @ k, t - rr @ k
        def y_of(uu, vv, a, b):
            un, vn = nn @ uu, nn @ vv
            da = response.interp(a, ts / dt, p) - response.interp(a, tr / dt, p)
            db = response.interp(b, ts / dt, p) - response.interp(b, tr / dt, p)
            return ((un * un - vn * vn) * da + 2 * un * vn * db) / (2 * (1 - nn @ k))
        y1 = response.link_response(hp, hc, 0.0, dt, "kepler", link, beta, lam, idx, p)
        assert np.allclose(y1, y_of(u, v, hp, hc), rtol=0, atol=1e-14 * np.max(np.abs(y1)))
        assert np.allclose(y1, y_of(u2, v2, hp2, hc2), rtol=0, atol=1e-12 * np.max(np.abs(y1)))


def test_source_basis_orthonormal_and_k_points_from_source():
    k, u, v = response.source_basis(-0.6, 0.6)
    M = np.stack([k, u, v])
    assert np.allclose(M @ M.T, np.eye(3), atol=1e-15)
    # k is the propagation direction: opposite to the sky position (beta, lambda)
    sky = np.array([math.cos(-0.6) * math.cos(0.6), math.cos(-0.6) * math.sin(0.6), math.sin(-0.6)])
    assert np.allclose(k, -sky)


def test_aet_special_combinations():
    X = np.array([1.0, 2.0]); Y = X.copy(); Z = X.copy()
    A, E, T = response.aet_from_xyz(X, Y, Z)
    assert np.allclose(A, 0) and np.allclose(E, 0) and np.allclose(T, math.sqrt(3) * X)
    A, E, T = response.aet_from_xyz(X, 0 * X, -X)       # X = -Z, Y = 0
    assert np.allclose(A, -math.sqrt(2) * X) and np.allclose(E, 0) and np.allclose(T, 0)


# ------------------------------------------------ nested delay operators ---
@pytest.mark.parametrize("gen", [15, 20])
def test_nested_chains_are_the_printed_terms(gen):
    """Each operator chain carries the link, sign and multiset of light times
    of the printed term it stands for (Sec. II.B, X_1.5 and X_2)."""
    printed = response.X15_TERMS if gen == 15 else response.X20_TERMS
    chains = response.X15_CHAINS if gen == 15 else response.X20_CHAINS
    assert len(chains) == len(printed)
    for (l, s, d), (lc, sc, c) in zip(printed, chains):
        assert (l, s, sorted(d)) == (lc, sc, sorted(c))
    for ch in range(3):
        for (l, s, d), (lc, sc, c) in zip(response.channel_terms(gen, ch),
                                          response.channel_terms(gen, ch, nested=True)):
            assert (l, s, sorted(d)) == (lc, sc, sorted(c))


@pytest.mark.parametrize("orbit", ["rigid", "static_kepler"])
def test_nested_delays_equal_sums_for_constant_arms(orbit):
    t = np.linspace(0.0, 5e6, 50)
    for gen in (15, 20):
        for ch in range(3):
            a = response.term_delays(orbit, gen, ch, t)
            b = response.term_delays(orbit, gen, ch, t, nested=True)
            for (l, s, D), (lb, sb, Db) in zip(a, b):
                assert (l, s) == (lb, sb)
                assert np.max(np.abs(D - Db)) <= 1e-13


def _laser_xyz(gen, nested, t, lasers):
    """X, Y, Z of pure laser noise, one laser p_k per craft, evaluated exactly:
    y_l(t) = p_s(t - L_l(t)) - p_r(t) for link l from s to r.  Each laser phase
    is taken as its phase at the output time t plus 2 pi f u for the (small)
    offset u (angle-addition formula), so that FP64 rounding of the large
    phase at t (~1e-10 rad at 5e6 s) is common to all terms and cancels."""
    def p(k, u):
        out = 0.0
        for (a, f, ph) in lasers[k]:
            base = 2 * math.pi * f * t + ph
            out = out + a * (np.sin(base) * np.cos(2 * math.pi * f * u)
                             + np.cos(base) * np.sin(2 * math.pi * f * u))
        return out

    def y(link, u):
        s, r = orbits.LINK_ENDS[link]
        return p(s, u - orbits.light_time("kepler", link, t + u)) - p(r, u)

    out = []
    for ch in range(3):
        acc = np.zeros(t.shape)
        for (link, sign, D) in response.term_delays("kepler", gen, ch, t, nested):
            acc = acc + sign * y(link, -D)
        out.append(acc)
    return out


def test_tdi2_nested_operators_cancel_laser_noise():
    """The defining property of second-generation TDI: with the delays applied
    as nested operators on flexing (Keplerian) arms, laser noise cancels to
    first order in the arm rates, so the residual is FP64 rounding of O(1)
    samples.  The printed commuting sums, and X_1.5 even with nested delays,
    leave a residual ~ p' L dL/dt ~ 1e-7 for dL/dt ~ 3e-9 (a wrong chain
    order, sign or evaluation time fails the first bound)."""
    rng = np.random.default_rng(11)
    lasers = {k: [(rng.uniform(0.5, 1.0), rng.uniform(1e-3, 2e-2), rng.uniform(0, 2 * math.pi))
                  for _ in range(4)] for k in (1, 2, 3)}
    t = np.linspace(200.0, 60 * 86400.0, 120)
    r2n = max(np.max(np.abs(v)) for v in _laser_xyz(20, True, t, lasers))
    r2c = max(np.max(np.abs(v)) for v in _laser_xyz(20, False, t, lasers))
    r15n = max(np.max(np.abs(v)) for v in _laser_xyz(15, True, t, lasers))
    assert r2n < 2e-12
    assert r2c > 1e-9 and r15n > 1e-9
    assert r2n < 1e-4 * min(r2c, r15n)
