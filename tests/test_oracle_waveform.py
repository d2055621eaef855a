"""Pins of the oracle's waveform stand-in, Wigner matrices, spherical
harmonics and two-step twist-up (Sec. II.A)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import consts as K
from oracle import waveform
from oracle.wigner import sYlm, small_d, wigner_D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rot(alpha, beta, gamma):
    def Rz(a):
        c, s = math.cos(a), math.sin(a)
        return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])

    def Ry(b):
        c, s = math.cos(b), math.sin(b)
        return np.array([[c, 0, s], [0, 1.0, 0], [-s, 0, c]])
    return Rz(alpha) @ Ry(beta) @ Rz(gamma)


def _euler(R):
    beta = math.acos(max(-1.0, min(1.0, R[2, 2])))
    alpha = math.atan2(R[1, 2], R[0, 2])
    gamma = math.atan2(R[2, 1], -R[2, 0])
    return alpha, beta, gamma


def _Dmat(l, a, b, g):
    ms = range(-l, l + 1)
    return np.array([[wigner_D(l, mp, m, a, b, g) for m in ms] for mp in ms])


# ------------------------------------------------------------ harmonics ----
def test_m2Y22_closed_form():
    th, ph = 0.83, 2.1
    want = math.sqrt(5 / (64 * math.pi)) * (1 + math.cos(th)) ** 2 * np.exp(2j * ph)
    assert abs(sYlm(-2, 2, 2, th, ph) - want) < 1e-15


def test_m2Y_special_values_l2():
    th = 1.1
    # textbook: -2Y_21 = sqrt(5/16pi) sin th (1 + cos th) e^{i phi}
    want = math.sqrt(5 / (16 * math.pi)) * math.sin(th) * (1 + math.cos(th))
    assert abs(sYlm(-2, 2, 1, th, 0.0) - want) < 1e-15
    # -2Y_2-2 = sqrt(5/64pi)(1 - cos th)^2 e^{-2 i phi}
    want = math.sqrt(5 / (64 * math.pi)) * (1 - math.cos(th)) ** 2
    assert abs(sYlm(-2, 2, -2, th, 0.0) - want) < 1e-15


@pytest.mark.parametrize("l", [2, 3, 4])
def test_m2Y_orthonormal_by_quadrature(l):
    x, wx = np.polynomial.legendre.leggauss(40)
    th = np.arccos(x)
    ph = np.linspace(0, 2 * math.pi, 64, endpoint=False)
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    W = wx[:, None] * (2 * math.pi / 64)
    ms = list(range(-l, l + 1))
    Y = [sYlm(-2, l, m, TH, PH) for m in ms]
    G = np.array([[np.sum(W * a * np.conj(b)) for b in Y] for a in Y])
    assert np.allclose(G, np.eye(len(ms)), atol=1e-12)


@pytest.mark.parametrize("l,m", [(2, 2), (2, -1), (3, 3), (3, -2), (4, 4), (4, 0)])
def test_m2Y_equals_wigner_d_relation(l, m):
    th, ph = 2.3, -0.7
    want = math.sqrt((2 * l + 1) / (4 * math.pi)) * np.exp(1j * m * ph) * small_d(l, m, 2, th)
    assert abs(sYlm(-2, l, m, th, ph) - want) < 1e-14


# --------------------------------------------------------------- Wigner ----
@pytest.mark.parametrize("l", [2, 3, 4])
def test_wigner_identity_unitarity_and_representation(l):
    assert np.allclose(_Dmat(l, 0, 0, 0), np.eye(2 * l + 1), atol=1e-15)
    rng = np.random.default_rng(l)
    a1, b1, g1, a2, b2, g2 = rng.uniform(0, math.pi, 6)
    D1, D2 = _Dmat(l, a1, b1, g1), _Dmat(l, a2, b2, g2)
    assert np.allclose(D1 @ D1.conj().T, np.eye(2 * l + 1), atol=1e-13)
    a, b, g = _euler(_rot(a1, b1, g1) @ _rot(a2, b2, g2))
    assert np.allclose(_Dmat(l, a, b, g), D1 @ D2, atol=1e-12)


def test_wigner_small_d_limits():
    for l in (2, 3, 4):
        for mp in range(-l, l + 1):
            for m in range(-l, l + 1):
                assert abs(small_d(l, mp, m, 0.0) - (1.0 if mp == m else 0.0)) < 1e-15
                want = (-1.0) ** (l - m) if mp == -m else 0.0
                assert abs(small_d(l, mp, m, math.pi) - want) < 1e-14
    # textbook d^1 entries
    b = 0.77
    assert abs(small_d(1, 1, 0, b) + math.sin(b) / math.sqrt(2)) < 1e-15
    assert abs(small_d(1, 0, 0, b) - math.cos(b)) < 1e-15


# ------------------------------------------------------------ stand-in -----
THETA_AL = np.array([6.667e5, 3.333e5, 0.5, 0, 0, 0.3, 0, 0, 20.0, 1.0, 0.7, 0.3, 1.2, 0.4,
                     0.75 * 86400])


def test_phase_derivative_is_frequency():
    src = waveform.source(THETA_AL, False)
    t = np.linspace(src["tm"] - 2e4, src["tm"] - 10.0, 50)
    h = 1e-2
    x = lambda tt: src["nu"] * (src["tc"] - tt) / (5 * src["M"])
    om, _ = waveform._omega_phase(src, x(t) ** 0.125)
    _, pp = waveform._omega_phase(src, x(t + h) ** 0.125)
    _, pm = waveform._omega_phase(src, x(t - h) ** 0.125)
    assert np.allclose((pp - pm) / (2 * h), om, rtol=1e-7)


def test_mode_c1_continuity_at_merger():
    src = waveform.source(THETA_AL, False)
    tm = src["tm"]
    for (l, m) in K.MODES:
        eps = 1e-4
        t = np.array([tm - 2 * eps, tm - eps, tm, tm + eps, tm + 2 * eps])
        h = waveform.mode(src, l, m, t, 0.0)
        amp = np.abs(h)
        ph = np.unwrap(-np.angle(h))
        if amp[2] == 0:
            continue
        left = (amp[1] - amp[0]) / eps, (ph[1] - ph[0]) / eps
        right = (amp[4] - amp[3]) / eps, (ph[4] - ph[3]) / eps
        assert abs(amp[3] - amp[1]) < 1e-6 * amp[2]
        assert abs(left[0] - right[0]) < 1e-3 * abs(left[0]) + 1e-12 * amp[2]
        assert abs(left[1] - right[1]) < 1e-3 * abs(left[1])


def test_amplitude_inverse_distance_and_zero_distance_limit():
    t = np.linspace(0, 86400, 200)
    a = waveform.plus_cross(THETA_AL, t, 0.0, 31, False)
    th2 = THETA_AL.copy()
    th2[8] *= 4
    b = waveform.plus_cross(th2, t, 0.0, 31, False)
    assert np.allclose(a[0], 4 * b[0], rtol=1e-14, atol=0)
    th2[8] = np.inf
    c = waveform.plus_cross(th2, t, 0.0, 31, False)
    assert np.all(c[0] == 0) and np.all(c[1] == 0)


def test_equal_mass_kills_odd_m_modes():
    th = THETA_AL.copy()
    th[0] = th[1] = 5e5
    src = waveform.source(th, False)
    t = np.linspace(0, 86400, 100)
    assert np.all(waveform.mode(src, 2, 1, t, 0.0) == 0)
    assert np.all(waveform.mode(src, 3, 3, t, 0.0) == 0)


def test_face_on_22_is_circular():
    th = THETA_AL.copy()
    th[9] = 0.0
    t = np.linspace(3e4, 6e4, 300)
    hp, hc = waveform.plus_cross(th, t, 0.0, 1, False)
    src = waveform.source(th, False)
    amp = np.abs(waveform.mode(src, 2, 2, t, 0.0)) * math.sqrt(5 / (4 * math.pi))
    assert np.allclose(np.hypot(hp, hc), amp, rtol=1e-12)


def test_polarisation_angle_rotation():
    t = np.linspace(3e4, 6e4, 100)
    th = THETA_AL.copy()
    th[13] = 0.0
    hp0, hc0 = waveform.plus_cross(th, t, 0.0, 31, False)
    th[13] = 0.3
    hp, hc = waveform.plus_cross(th, t, 0.0, 31, False)
    # (h+ - i hx) -> (h+ - i hx) e^{2 i psi}
    z = (hp0 - 1j * hc0) * np.exp(0.6j)
    assert np.allclose(hp, z.real, atol=1e-14 * np.max(np.abs(hp0)))
    assert np.allclose(hc, -z.imag, atol=1e-14 * np.max(np.abs(hp0)))


def test_start_taper_and_window_start():
    th = THETA_AL.copy()
    t = np.array([0.0, 1.0, K.T_TAPER * 0.5, K.T_TAPER + 1.0])
    src = waveform.source(th, False)
    h = waveform.mode(src, 2, 2, t, 0.0)
    assert h[0] == 0 and 0 < abs(h[1]) < abs(h[2]) < abs(h[3])


def test_high_frequency_taper_removes_light_ringdowns():
    th = THETA_AL.copy()
    th[0], th[1] = 6e4, 4e4                 # M = 1e5 Msun: ringdown far above 0.09 Hz
    src = waveform.source(th, False)
    t = np.linspace(src["tm"] + 1.0, src["tm"] + 200.0, 50)
    assert np.all(waveform.mode(src, 2, 2, t, 0.0) == 0)


# ------------------------------------------------------------ precession ---
THETA_PR = np.array([1.0e6, 0.7e6, 0.7, math.radians(40.1), math.radians(40.1), 0.4,
                     math.radians(22.9), math.radians(22.9), 20.0, math.radians(149.0),
                     math.radians(229.2), math.radians(-34.4), math.radians(34.4),
                     math.radians(22.9), 0.9 * 61 * 86400])


def test_euler_angle_rates():
    src = waveform.source(THETA_PR, True)
    t = np.linspace(src["tm"] - 3e5, src["tm"] - 100, 40)
    h = 0.05
    a0, b0, g0, _ = waveform.euler_angles(src, t)
    ap, _, gp, _ = waveform.euler_angles(src, t + h)
    am, _, gm, _ = waveform.euler_angles(src, t - h)
    M, nu = src["M"], src["nu"]
    u = (nu * (src["tc"] - t) / (5 * M)) ** 0.125
    S = src["a1"] * (src["m1"] / (src["m1"] + src["m2"])) ** 2
    L = 2 * nu * u
    J = np.sqrt(L ** 2 + 2 * L * S * math.cos(src["tilt1"]) + S ** 2)
    adot = (2 + 1.5 * src["m2"] / src["m1"]) * J * (u ** -3 / 8) ** 2 / M
    assert np.allclose((ap - am) / (2 * h), adot, rtol=1e-6)
    assert np.allclose((gp - gm) / (2 * h), -np.cos(b0) * adot, rtol=1e-6)
    assert np.allclose(np.cos(b0), (L + S * math.cos(src["tilt1"])) / J, rtol=1e-13)


def test_precessing_without_spin_equals_aligned():
    th = THETA_PR.copy()
    th[2] = 0.0                              # no in-plane or aligned spin-1
    t = np.linspace(4.6e6, 4.75e6, 300)
    hp, hc = waveform.plus_cross(th, t, 0.0, 31, True)
    al = th.copy()
    al[5] = th[5] * math.cos(th[6])          # chi2 = a2 cos(theta2) on the aligned model
    hpa, hca = waveform.plus_cross(al, t, 0.0, 31, False)
    scale = np.max(np.abs(hpa))
    assert np.max(np.abs(hp - hpa)) < 1e-12 * scale
    assert np.max(np.abs(hc - hca)) < 1e-12 * scale


def test_two_step_equals_single_rotation_sum():
    """The two sums of the twist-up collapse to one sum over the composed
    rotation (the identity behind the single-sum form, Eq. newtwistup)."""
    src = waveform.source(THETA_PR, True)
    t = np.array([src["tm"] - 5e4])
    al, be, ga, rot0 = waveform.euler_angles(src, t)
    Rt = _rot(*rot0) @ _rot(al[0], be[0], ga[0])
    a, b, g = _euler(Rt)

    def Dp(l, *ang):
        ms = range(-l, l + 1)
        return np.array([[waveform.paper_D(l, m, mp, *ang) for mp in ms] for m in ms])
    for l in (2, 3, 4):
        two = Dp(l, *rot0).conj() @ Dp(l, al[0], be[0], ga[0]).conj()
        assert np.allclose(two, Dp(l, a, b, g).conj(), atol=1e-12)


def test_reference_frame_at_reference_time_is_identity():
    src = waveform.source(THETA_PR, True)
    M = src["M"]
    u_ref = (8 * math.pi * M * K.F_MIN) ** (-1 / 3)
    t_ref = src["tc"] - 5 * M * u_ref ** 8 / src["nu"]
    al, be, ga, rot0 = waveform.euler_angles(src, np.array([t_ref]))
    assert abs(al[0]) < 1e-9
    R = _rot(*rot0) @ _rot(al[0], be[0], ga[0])
    assert np.allclose(R, np.eye(3), atol=1e-9)


def test_table1_injection_runs_and_is_finite():
    with open(os.path.join(GOLDEN, "table1_injection.json")) as f:
        g = json.load(f)
    th = np.array(g["precessing_theta"], dtype=float)
    th[14] = 0.9 * g["duration_days"] * 86400
    t = np.linspace(0, g["duration_days"] * 86400, 2000)
    hp, hc = waveform.plus_cross(th, t, 0.0, 31, True)
    assert np.all(np.isfinite(hp)) and np.max(np.abs(hp)) > 0
    assert g["dt_s"] == 10.0 and g["snr_approx"] == 2800


# ------------------------------------- twist-up against 3-vector geometry ----
def _spherical_basis(n):
    """Polar angles of the unit vector n and the tangent vectors e_theta, e_phi there."""
    th = math.acos(max(-1.0, min(1.0, n[2])))
    ph = math.atan2(n[1], n[0])
    e_th = np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)])
    e_ph = np.array([-math.sin(ph), math.cos(ph), 0.0])
    return th, ph, e_th, e_ph


def _strain_seen_through_rotation(cp_modes, M, iota, phi):
    """h+, hx along the direction (iota, phi) of the L0 frame when the source's
    co-precessing frame has axes M e_x, M e_y, M e_z in L0 coordinates.

    No Wigner matrix enters: the line of sight and its polarisation basis are
    carried into the co-precessing frame by the 3x3 matrix M^T, the strain is
    the mode sum h+ - i hx = sum h_lm -2Y_lm there, rebuilt as the transverse
    tensor h+(e_th e_th - e_ph e_ph) + hx(e_th e_ph + e_ph e_th), and projected
    back onto the carried basis."""
    n0 = np.array([math.sin(iota) * math.cos(phi), math.sin(iota) * math.sin(phi), math.cos(iota)])
    _, _, a0, b0 = _spherical_basis(n0)
    n, a, b = M.T @ n0, M.T @ a0, M.T @ b0
    th, ph, e_th, e_ph = _spherical_basis(n)
    H = sum(h * sYlm(-2, l, m, th, ph) for (l, m), h in cp_modes.items())
    hp, hx = H.real, -H.imag
    T = (hp[:, None, None] * (np.outer(e_th, e_th) - np.outer(e_ph, e_ph))
         + hx[:, None, None] * (np.outer(e_th, e_ph) + np.outer(e_ph, e_th)))
    plus = 0.5 * (np.einsum("i,tij,j->t", a, T, a) - np.einsum("i,tij,j->t", b, T, b))
    cross = np.einsum("i,tij,j->t", a, T, b)
    return plus, cross


@pytest.mark.parametrize("angles,rot0", [
    ((0.7, 0.3, -1.1), (0.0, 0.0, 0.0)),
    ((-2.0, math.pi / 2, 0.4), (0.0, 0.0, 0.0)),
    ((1.3, math.pi - 0.2, 2.2), (0.0, 0.0, 0.0)),
    ((0.9, 0.0, -0.35), (0.0, 0.0, 0.0)),            # pure z-rotation
    ((0.7, 0.3, -1.1), (2.5, -0.45, 0.0)),           # both rotations generic
    ((-0.6, 1.9, 0.8), (-1.2, -1.3, 0.6)),
])
def test_twist_up_is_the_rotation_of_the_emission_pattern(monkeypatch, angles, rot0):
    """The two-step twist-up of ``plus_cross`` (Sec. II.A, the two sums of D*
    and the sum with -2Y) must equal what plain 3-vector geometry gives for a
    co-precessing frame whose axes are R(alpha,beta,gamma) = Rz(alpha)Ry(beta)Rz(gamma)
    applied to the J axes (so L points at polar angle beta, azimuth alpha in
    the J frame), and a J -> L0 map R(rot0).  The Euler angles are frozen to
    constants so the identity holds sample by sample; a Wigner D in place of
    D*, swapped indices or the inverse rotation each break it."""
    th = np.array(THETA_PR, dtype=float)
    th[13] = 0.0                                     # no polarisation rotation
    src = waveform.source(th, True)
    t = np.linspace(src["tm"] - 4e4, src["tm"] + 200.0, 64)

    def frozen(src_, t_):
        one = np.ones(np.shape(t_))
        return angles[0] * one, angles[1] * one, angles[2] * one, rot0
    monkeypatch.setattr(waveform, "euler_angles", frozen)
    hp, hx = waveform.plus_cross(th, t, 0.0, 31, True)

    cp = {}
    for (l, m) in K.MODES:
        h = waveform.mode(src, l, m, t, 0.0)
        cp[(l, m)] = h
        cp[(l, -m)] = (-1.0) ** l * np.conj(h)
    M = _rot(*rot0) @ _rot(*angles)
    gp, gx = _strain_seen_through_rotation(cp, M, src["iota"], src["phi_ref"])
    scale = max(np.max(np.abs(gp)), np.max(np.abs(gx)))
    assert scale > 0
    assert np.max(np.abs(hp - gp)) < 1e-12 * scale
    assert np.max(np.abs(hx - gx)) < 1e-12 * scale


def test_geometric_strain_reduces_to_mode_sum_without_rotation():
    """With M = identity the geometric construction is the plain mode sum."""
    rng = np.random.default_rng(7)
    cp = {(l, m): rng.normal(size=5) + 1j * rng.normal(size=5)
          for l in (2, 3) for m in range(-l, l + 1)}
    iota, phi = 1.1, -0.4
    gp, gx = _strain_seen_through_rotation(cp, np.eye(3), iota, phi)
    H = sum(h * sYlm(-2, l, m, iota, phi) for (l, m), h in cp.items())
    assert np.allclose(gp, H.real, atol=1e-14) and np.allclose(gx, -H.imag, atol=1e-14)
