"""Pins of the oracle's orbit models (Sec. II.B) and likelihood stage
(DFT, PSD, inner product, logL; Sec. II.B end)."""
import math

import numpy as np
import pytest

from oracle import consts as K
from oracle import likelihood, orbits, pipeline

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ----------------------------------------------------------------- orbits --
def test_rigid_triangle_geometry():
    t = np.linspace(0, 3e7, 7)
    r = [orbits.rigid_position(k, t) for k in (1, 2, 3)]
    for i in range(3):
        d = np.linalg.norm(r[i] - r[(i + 1) % 3], axis=-1)
        assert np.allclose(d, K.ARM_S, rtol=1e-14)
    c = (r[0] + r[1] + r[2]) / 3
    assert np.allclose(np.linalg.norm(c, axis=-1), K.AU_S, rtol=1e-14)
    nrm = np.cross(r[1] - r[0], r[2] - r[0])
    cosang = np.abs(nrm[:, 2]) / np.linalg.norm(nrm, axis=-1)
    assert np.allclose(cosang, 0.5, atol=1e-12)          # plane at 60 deg to ecliptic


def test_kepler_orbits():
    t = np.linspace(0, 3.2e7, 50)
    for k in (1, 2, 3):
        e = K.KEPLER_E0 * (1 + K.KEPLER_ETA[k - 1])
        r = np.linalg.norm(orbits.kepler_position(k, t), axis=-1)
        assert np.all(r <= K.AU_S * (1 + e) * (1 + 1e-14))
        assert np.all(r >= K.AU_S * (1 - e) * (1 - 1e-14))
    M = np.linspace(-3, 9, 101)
    E = orbits._solve_kepler(M, 0.3)
    assert np.max(np.abs(E - 0.3 * np.sin(E) - M)) < 1e-14
    # nearly rigid: arms within 1.5% of the nominal light time, but breathing
    for l in orbits.LINKS:
        L = orbits.light_time("kepler", l, t)
        assert np.all(np.abs(L / K.ARM_S - 1) < 0.015)
        assert np.ptp(L) > 1e-4


def test_light_time_solves_light_cone_equation():
    t = np.linspace(1e5, 3e7, 9)
    for l in orbits.LINKS:
        s, r = orbits.LINK_ENDS[l]
        L = orbits.light_time("kepler", l, t)
        res = np.linalg.norm(orbits.position("kepler", r, t)
                             - orbits.position("kepler", s, t - L), axis=-1) - L
        assert np.max(np.abs(res)) < 1e-12
    # opposite directions of a moving arm differ (Sagnac-like), as they must
    assert np.max(np.abs(orbits.light_time("kepler", 1, t) - orbits.light_time("kepler", -1, t))) > 1e-6


# -------------------------------------------------------------------- DFT --
@pytest.mark.parametrize("n", [60, 120, 840, 17280, 244, 3904, 19520])   # 244, 3904, 19520: the factor 61 of the 61-day grid
def test_fft_matches_bruteforce_dft(n):
    rng = np.random.default_rng(n)
    a = rng.normal(size=n)
    if n > 2000:
        sel = np.arange(0, n // 2 + 1, 97)
        j = np.arange(n)
        brute = np.array([5.0 * np.sum(a * np.exp(-2j * math.pi * ((k * j) % n) / n)) for k in sel])
        assert np.allclose(likelihood.dft(a, 5.0)[sel], brute, atol=1e-9 * np.sqrt(n))
    else:
        assert np.allclose(likelihood.dft(a, 5.0), likelihood.dft_brute(a, 5.0), atol=1e-11 * n)


def test_parseval_and_white_noise_inner_product():
    rng = np.random.default_rng(1)
    n, dt = 840, 5.0
    a, b = rng.normal(size=n), rng.normal(size=n)
    A, B = likelihood.dft(a, dt), likelihood.dft(b, dt)
    two_sided = np.sum(np.abs(A) ** 2) * 2 - np.abs(A[0]) ** 2 - np.abs(A[-1]) ** 2
    assert math.isclose(two_sided, dt * dt * n * np.sum(a * a), rel_tol=1e-12)
    # white PSD, full band with half weights at DC / Nyquist: (a|b) = 2 dt sum a b / S
    S = 3.0
    w = np.ones(n // 2 + 1)
    w[0] = w[-1] = 0.5
    df = 1.0 / (n * dt)
    ip = 4 * df * np.sum(w * (A * np.conj(B)).real) / S
    assert math.isclose(ip, 2 * dt * np.sum(a * b) / S, rel_tol=1e-12)


# -------------------------------------------------------------------- PSD --
def test_psd_low_frequency_limits_and_tdi2_factor():
    f = np.array([1e-5, 2e-5])
    s_acc, s_op = likelihood.psd_components(f)
    x = 2 * math.pi * f * K.ARM_S
    s_ae, s_t = likelihood.psd_aet(f, 15)
    assert np.allclose(s_ae, x ** 2 * (96 * s_acc + 24 * s_op), rtol=1e-6)
    assert np.allclose(s_t, 8 * s_op * x ** 4 + 8 * s_acc * x ** 6, rtol=1e-6)
    f = np.array([3e-4, 3e-3, 1.7e-2])
    x = 2 * math.pi * f * K.ARM_S
    a15, t15 = likelihood.psd_aet(f, 15)
    a20, t20 = likelihood.psd_aet(f, 20)
    assert np.allclose(a20 / a15, 4 * np.sin(2 * x) ** 2, rtol=1e-13)
    assert np.allclose(t20 / t15, 4 * np.sin(2 * x) ** 2, rtol=1e-13)


def test_psd_noise_budget_scalings():
    # acceleration noise ~ f^-2 of fractional frequency at low f, OMS ~ f^-2 too
    # with a (1 + (2e-3/f)^4) knee; check exact ratios between two frequencies
    f1, f2 = 1e-2, 2e-2
    a1, o1 = likelihood.psd_components(np.array([f1]))
    a2, o2 = likelihood.psd_components(np.array([f2]))
    ra = ((1 + (4e-4 / f2) ** 2) * (1 + (f2 / 8e-3) ** 4)) / ((1 + (4e-4 / f1) ** 2) * (1 + (f1 / 8e-3) ** 4))
    assert math.isclose(a2[0] / a1[0], ra * (f2 / f1) ** -2, rel_tol=1e-12)
    ro = (1 + (2e-3 / f2) ** 4) / (1 + (2e-3 / f1) ** 4)
    assert math.isclose(o2[0] / o1[0], ro * (f2 / f1) ** 2, rel_tol=1e-12)
    # the A_acc reading puts the acceleration and OMS terms near each other at ~3 mHz
    a, o = likelihood.psd_components(np.array([3e-3]))
    assert 0.01 < a[0] / o[0] < 100


# ------------------------------------------------------------------- logL --
def _small_setup():
    return pipeline.Setup(n=2880, orbit="rigid", tdi_gen=15, mode_mask=1, lagrange_order=7,
                          f_lo=1e-4, f_hi=0.02)


THETA = np.array([6.667e5, 3.333e5, 0.5, 0, 0, 0.3, 0, 0, 20.0, 1.0, 0.7, 0.3, 1.2, 0.4, 0.1 * 86400])


def test_zero_noise_loglike_is_zero_at_truth_and_quadratic():
    s = _small_setup()
    d = pipeline.aet(THETA, s)
    assert pipeline.loglike(THETA, s, d) == 0.0
    dd = -2 * likelihood.loglike(np.zeros_like(d), d, s.dt, s.f_lo, s.f_hi, 15)
    assert dd > 0
    for eps in (0.5, -0.25):
        ll = likelihood.loglike((1 + eps) * d, d, s.dt, s.f_lo, s.f_hi, 15)
        assert math.isclose(ll, -0.5 * eps * eps * dd, rel_tol=1e-12)
    th = THETA.copy()
    th[12] += 0.01
    assert pipeline.loglike(th, s, d) < 0


def test_channel_mask_monotone():
    s = _small_setup()
    d = pipeline.aet(THETA, s)
    z = np.zeros_like(d)
    vals = [likelihood.loglike(z, d, s.dt, s.f_lo, s.f_hi, 15, m) for m in (1, 3, 7)]
    assert vals[0] > vals[1] > vals[2]
    a = likelihood.loglike(z, d, s.dt, s.f_lo, s.f_hi, 15, 1)
    e = likelihood.loglike(z, d, s.dt, s.f_lo, s.f_hi, 15, 2)
    assert math.isclose(a + e, vals[1], rel_tol=1e-13)


def test_band_limits():
    m = likelihood.band(1000, 5.0, 1e-4, 0.02)
    f = likelihood.freqs(1000, 5.0)
    assert not m[0] and not m[-1]
    assert np.all(f[m] >= 1e-4) and np.all(f[m] <= 0.02)
    assert m.sum() == np.sum((f >= 1e-4) & (f <= 0.02))


# ------------------------------------------------------ orbit tables --------
def test_orbit_table_interpolation_is_exact_for_degree_seven_paths():
    """The table's resampling is the degree-7 Lagrange polynomial through eight
    rows: it reproduces trajectories that are polynomials of degree <= 7 in
    time to rounding (near the ends too, where the eight rows move inwards),
    and no longer does at degree 8."""
    rng = np.random.default_rng(11)
    t0, dt, rows = -7200.0, 3600.0, 40
    tt = t0 + dt * np.arange(rows)
    ts = np.concatenate([rng.uniform(t0, tt[-1], 200), [t0, t0 + 0.3 * dt, tt[-1] - 0.2 * dt]])
    c = rng.normal(size=(8, 3, 3)) * 1e9

    def path(t):
        x = (np.asarray(t) - t0) / (rows * dt)
        return sum(c[d] * x[..., None, None] ** d for d in range(8))
    tab = orbits.OrbitTable(t0, dt, path(tt))
    for k in (1, 2, 3):
        want = path(ts)[:, k - 1, :] / K.C_SI
        err = np.max(np.abs(tab.position(k, ts) - want)) / np.max(np.abs(want))
        assert err < 1e-12, (k, err)
    # x^8 on one stencil's rows: the error at the middle is prod (3.5 - k) = 43
    # against a largest value of 7^8
    p8 = np.zeros((8, 3, 3))
    p8[:, 0, 0] = np.arange(8.0) ** 8
    got = orbits.OrbitTable(0.0, dt, p8).position(1, np.array([3.5 * dt]))[0, 0] * K.C_SI
    assert abs(got - 3.5 ** 8) == pytest.approx(43.06640625, rel=1e-9)


def test_orbit_table_of_keplerian_positions_reproduces_the_keplerian_model():
    """Keplerian positions tabulated hourly and resampled through the table:
    positions, light times and A, E, T of a source agree with the analytic
    Keplerian model to the interpolant's error (Omega dt ~ 7e-4 rad per row)."""
    t0, dt = -3 * 3600.0, 3600.0
    rows = 12
    tt = t0 + dt * np.arange(rows)
    pos = np.stack([orbits.kepler_position(k, tt) for k in (1, 2, 3)], axis=1) * K.C_SI
    tab = orbits.OrbitTable(t0, dt, pos)
    ts = np.linspace(0.0, 4 * 3600.0, 77)
    for k in (1, 2, 3):
        assert np.max(np.abs(tab.position(k, ts) - orbits.kepler_position(k, ts))) < 1e-9
    for l in orbits.LINKS:
        assert np.max(np.abs(orbits.light_time(tab, l, ts) - orbits.light_time("kepler", l, ts))) < 1e-11
    th = np.array([6e5, 3e5, 0.4, 0, 0, -0.2, 0, 0, 3.0, 0.7, 1.1, 0.3, 2.0, 0.4, 2.5 * 3600.0])
    sk = pipeline.Setup(n=2880, tdi_gen=20, orbit="kepler", mode_mask=31)
    st = pipeline.Setup(n=2880, tdi_gen=20, orbit=tab, mode_mask=31)
    a, b = pipeline.aet(th, sk), pipeline.aet(th, st)
    assert np.max(np.abs(a - b)) <= 1e-9 * np.max(np.abs(a))
