"""Declared stand-in for the IMRPhenomT family (Sec. II.A) and the two-step
twist-up of its precessing members (Sec. II.A, the three displayed equations
h^J = sum D* h^CP, h^L0 = sum D* h^J, h+ - i hx = sum h^L0 -2Y).

Reading of the twist-up (the paper does not fix its Wigner-D phase
convention): the paper's D^l_{m m'}(alpha, beta, gamma) is taken as
e^{+i m alpha} d^l_{m m'}(beta) e^{+i m' gamma}, the complex conjugate of the
textbook ``wigner.wigner_D``.  With it the printed sums of D* rotate the
co-precessing frame by R(alpha, beta, gamma) = Rz(alpha) Ry(beta) Rz(gamma):
the CP axes are R applied to the J axes, so L sits at polar angle beta and
azimuth alpha in the J frame.  The J -> L0 step is the rotation R(rot0).
Pinned against 3-vector geometry (rotating the line of sight and its
polarisation basis, no Wigner matrix) by
``test_twist_up_is_the_rotation_of_the_emission_pattern``.

The paper uses IMRPhenomT(HM)(P)(HM) but takes its coefficients from earlier
work; the stand-in keeps the same structure -- every time sample is an
independent closed form, modes (2,+-2),(2,+-1),(3,+-3),(3,+-2),(4,+-4),
h_{l,-m} = (-1)^l conj(h_{lm}) for the co-precessing / aligned modes -- with
the constants in ``consts``.  All formulas here are the definition of the
stand-in (FP64).

Parameter vector (15 entries, declared order; angles in radians):
  0 m1 [Msun]  1 m2 [Msun]  2 a1 (spin-1 magnitude, or chi1z when aligned)
  3 theta1  4 phi1  5 a2 (or chi2z)  6 theta2  7 phi2  8 D [Gpc]  9 iota
  10 phi_ref  11 beta (ecl. latitude)  12 lambda (ecl. longitude)  13 psi
  14 t_c [s] (time parameter of the inspiral closed form)
"""
import math

import numpy as np

from . import consts as K
from .wigner import sYlm, wigner_D

PARAM_NAMES = ("m1", "m2", "a1", "theta1", "phi1", "a2", "theta2", "phi2", "D",
               "iota", "phi_ref", "beta", "lambda", "psi", "t_c")


def modes_from_mask(mask):
    """(l, m>0) modes selected by bits 0..4 = (2,2),(2,1),(3,3),(3,2),(4,4)."""
    return [lm for b, lm in enumerate(K.MODES) if (mask >> b) & 1]


def source(theta, precessing):
    """Derived per-source constants (all FP64)."""
    th = [float(x) for x in theta]
    m1, m2 = th[0], th[1]
    s1, s2 = (th[2], th[3], th[4]), (th[5], th[6], th[7])
    if m2 > m1:                                   # declared: m1 >= m2 by swapping
        m1, m2, s1, s2 = m2, m1, s2, s1
    mt = m1 + m2
    M = mt * K.MTSUN_SI
    nu = m1 * m2 / mt ** 2
    delta = (m1 - m2) / mt
    if precessing:
        chi1, chi2 = s1[0] * math.cos(s1[1]), s2[0] * math.cos(s2[1])
    else:
        chi1, chi2 = s1[0], s2[0]
    chi = (m1 * chi1 + m2 * chi2) / mt
    src = dict(m1=m1, m2=m2, M=M, nu=nu, delta=delta, chi=chi,
               a1=s1[0], tilt1=s1[1], phi1=s1[2],
               D=th[8] * K.GPC_S, iota=th[9], phi_ref=th[10], beta=th[11],
               lam=th[12], psi=th[13], tc=th[14])
    src["c1"] = 743.0 / 2688.0 + 11.0 * nu / 32.0
    src["cs"] = K.C_SPIN * chi
    # attachment of the ringdown: x = X_MERGE
    src["um"] = K.X_MERGE ** 0.125
    src["tm"] = src["tc"] - 5.0 * M * K.X_MERGE / nu
    # final-spin stand-in and Berti-Cardoso-Will (2,2,0) fits
    af = 0.686 + 0.25 * chi
    src["w_rd22"] = (1.5251 - 1.1568 * (1.0 - af) ** 0.1292) / M
    Q = 0.7 + 1.4187 * (1.0 - af) ** (-0.4990)
    src["tau_d"] = 2.0 * Q / src["w_rd22"]
    # start of the signal: Newtonian (2,2) frequency equals F_MIN
    u_s = (8.0 * math.pi * M * K.F_MIN) ** (-1.0 / 3.0)
    src["t_start"] = src["tc"] - 5.0 * M * u_s ** 8 / nu
    return src


def _omega_phase(src, u):
    """Orbital frequency omega(u) [rad/s] and phase phi(u) of the inspiral,
    u = x^(1/8), x = nu (t_c - t)/(5M).  phi is the exact integral of omega."""
    M, nu, c1, cs = src["M"], src["nu"], src["c1"], src["cs"]
    om = (u ** -3 + c1 * u ** -5 + cs * u ** -6) / (8.0 * M)
    ph = -(u ** 5 + (5.0 / 3.0) * c1 * u ** 3 + 2.5 * cs * u ** 2) / nu
    return om, ph


def _omega_dot(src, u):
    M, nu, c1, cs = src["M"], src["nu"], src["c1"], src["cs"]
    return ((3.0 * u ** -4 + 5.0 * c1 * u ** -6 + 6.0 * cs * u ** -7) / (8.0 * M)
            * nu * u ** -7 / (40.0 * M))


def _amp_coeff(src, l, m):
    """Leading-PN mode amplitude |h_lm| / [(M nu/D) 8 sqrt(pi/5) (M w)^(2/3)]
    as  coefficient * (M w)^(extra power / 3)."""
    nu, de = src["nu"], src["delta"]
    table = {(2, 2): (1.0, 0), (2, 1): (de / 3.0, 1),
             (3, 3): (0.75 * math.sqrt(15.0 / 14.0) * de, 1),
             (3, 2): (math.sqrt(5.0 / 7.0) * (1.0 - 3.0 * nu) / 3.0, 2),
             (4, 4): (8.0 / 9.0 * math.sqrt(5.0 / 7.0) * (1.0 - 3.0 * nu), 2)}
    return table[(l, m)]


def planck_rise(t, t_a, T):
    """Planck taper: 0 at t <= t_a, 1 at t >= t_a + T, smooth in between."""
    t = np.asarray(t, dtype=np.float64)
    out = np.where(t >= t_a + T, 1.0, 0.0)
    inside = (t > t_a) & (t < t_a + T)
    if np.any(inside):
        ti = t[inside]
        z = T / (ti - t_a) - T / (t_a + T - ti)
        out[inside] = 1.0 / (1.0 + np.exp(np.clip(z, -700.0, 700.0)))
    return out


def planck_fall_freq(f):
    """Per-mode high-frequency taper: 1 below F_HI_1, 0 above F_HI_2."""
    f = np.asarray(f, dtype=np.float64)
    out = np.where(f <= K.F_HI_1, 1.0, 0.0)
    inside = (f > K.F_HI_1) & (f < K.F_HI_2)
    if np.any(inside):
        fi = f[inside]
        d = K.F_HI_2 - K.F_HI_1
        z = d / (K.F_HI_2 - fi) - d / (fi - K.F_HI_1)
        out[inside] = 1.0 / (1.0 + np.exp(np.clip(z, -700.0, 700.0)))
    return out


def mode_phase(src, l, m, t):
    """Phase Phi_lm(t) and angular frequency of mode (l, m > 0), h_lm = A e^{-i Phi}:
    m phi(u) in the inspiral, the C1-continuous ringdown phase after t_m."""
    t = np.asarray(t, dtype=np.float64)
    M, nu = src["M"], src["nu"]
    um, tm, tau_d = src["um"], src["tm"], src["tau_d"]
    insp = t < tm
    x = np.where(insp, nu * (src["tc"] - t) / (5.0 * M), K.X_MERGE)
    u = x ** 0.125
    om, ph = _omega_phase(src, u)
    om_m, ph_m = _omega_phase(src, um)
    w_rd = K.RD_RATIO[(l, m)] * src["w_rd22"]
    tau = np.maximum(t - tm, 0.0)
    decay_f = np.exp(-tau / tau_d)
    phase_r = m * ph_m + w_rd * tau + (m * om_m - w_rd) * tau_d * (1.0 - decay_f)
    freq_r = w_rd + (m * om_m - w_rd) * decay_f
    return np.where(insp, m * ph, phase_r), np.where(insp, m * om, freq_r)


def mode(src, l, m, t, t0):
    """Complex mode h_lm(t) (m > 0) of the aligned / co-precessing stand-in."""
    t = np.asarray(t, dtype=np.float64)
    M, nu, D = src["M"], src["nu"], src["D"]
    um, tm, tau_d = src["um"], src["tm"], src["tau_d"]
    coef, extra = _amp_coeff(src, l, m)
    pref = M * nu / D * 8.0 * math.sqrt(math.pi / 5.0) * coef
    p = (2.0 + extra) / 3.0                      # A_lm ~ (M w)^p

    insp = t < tm
    x = np.where(insp, nu * (src["tc"] - t) / (5.0 * M), K.X_MERGE)
    u = x ** 0.125
    om, _ = _omega_phase(src, u)
    amp_i = pref * (M * om) ** p

    # ringdown, C1-continuous at t_m
    om_m, _ = _omega_phase(src, um)
    A_m = pref * (M * om_m) ** p
    a_lm = p * _omega_dot(src, um) / om_m + 1.0 / tau_d
    tau = np.maximum(t - tm, 0.0)
    decay_f = np.exp(-tau / tau_d)
    amp_r = A_m * (1.0 + a_lm * tau) * decay_f

    amp = np.where(insp, amp_i, amp_r)
    phase, freq = mode_phase(src, l, m, t)
    t_a = max(t0, src["t_start"])
    win = np.where(t >= src["t_start"], planck_rise(t, t_a, K.T_TAPER), 0.0)
    win = win * planck_fall_freq(freq / (2.0 * math.pi))
    return amp * win * np.exp(-1j * phase)


# ---------------------------------------------------------------------------
# precession stand-in (single-spin simple precession, closed forms)
# ---------------------------------------------------------------------------

def euler_angles(src, t):
    """alpha, beta, gamma of the co-precessing -> J rotation at times t.

    Declared model: L = nu (M w_N)^(-1/3) = 2 nu u with the Newtonian w_N,
    S = a1 (m1/M)^2 at tilt theta1; J = L + S; cos beta = (L + S cos th1)/|J|;
    d alpha/dt = (2 + 1.5 m2/m1) |J| (M w_N)^2 / M;  d gamma/dt = -cos(beta) d alpha/dt
    (minimal rotation).  Both integrate in closed form in u; alpha(t_ref) = 0,
    gamma(t_ref) = pi - phi1 with t_ref where the Newtonian (2,2) frequency is
    F_MIN.  Frozen for t >= t_m."""
    t = np.asarray(t, dtype=np.float64)
    M, nu = src["M"], src["nu"]
    S = src["a1"] * (src["m1"] / (src["m1"] + src["m2"])) ** 2
    c, s = math.cos(src["tilt1"]), math.sin(src["tilt1"])
    b = S * s
    kp = 2.0 + 1.5 * src["m2"] / src["m1"]
    x = np.where(t < src["tm"], nu * (src["tc"] - t) / (5.0 * M), K.X_MERGE)
    u = x ** 0.125
    u_ref = (8.0 * math.pi * M * K.F_MIN) ** (-1.0 / 3.0)

    def G(a):
        r = np.sqrt(a * a + b * b)
        ash = np.arcsinh(a / b) if b > 0.0 else 0.0 * a
        return r ** 3 / 3.0 - S * c * (0.5 * a * r + 0.5 * b * b * ash)

    a_u = 2.0 * nu * u + S * c
    a_ref = 2.0 * nu * u_ref + S * c
    J = np.sqrt(a_u * a_u + b * b)
    cosb = a_u / J
    sinb = b / J
    beta = np.arctan2(sinb, cosb)
    alpha = -(5.0 * kp / (32.0 * nu ** 3)) * (G(a_u) - G(a_ref))
    gamma = (math.pi - src["phi1"]) + (5.0 * kp / (8.0 * nu)) * (
        2.0 * nu * (u ** 3 - u_ref ** 3) / 3.0 + 0.5 * S * c * (u ** 2 - u_ref ** 2))
    beta_ref = math.atan2(b / math.hypot(a_ref, b), a_ref / math.hypot(a_ref, b))
    rot0 = (src["phi1"] - math.pi, -beta_ref, 0.0)   # J -> L0 (inverse of R1(t_ref))
    return alpha, beta, gamma, rot0


def paper_D(l, m, mp, alpha, beta, gamma):
    """The Wigner-D of the twist-up equations (Sec. II.A) under the reading in
    the module docstring: e^{+i m alpha} d^l_{m mp}(beta) e^{+i mp gamma}."""
    return np.conj(wigner_D(l, m, mp, alpha, beta, gamma))


def plus_cross(theta, t, t0, mode_mask, precessing):
    """h+ and hx in the (u, v) frame after the polarisation rotation by psi:
    (h+ - i hx) -> (h+ - i hx) exp(2 i psi)  (Sec. III.A)."""
    src = source(theta, precessing)
    t = np.asarray(t, dtype=np.float64)
    lms = modes_from_mask(mode_mask)
    iota, phr = src["iota"], src["phi_ref"]
    hpc = np.zeros(t.shape, dtype=np.complex128)        # h+ - i hx
    if not precessing:
        for (l, m) in lms:
            h = mode(src, l, m, t, t0)
            hpc += h * sYlm(-2, l, m, iota, phr)
            hpc += (-1.0) ** l * np.conj(h) * sYlm(-2, l, -m, iota, phr)
    else:
        alpha, beta, gamma, rot0 = euler_angles(src, t)
        for l in sorted({lm[0] for lm in lms}):
            cp = {}
            for (ll, m) in lms:
                if ll != l:
                    continue
                h = mode(src, l, m, t, t0)
                cp[m] = h
                cp[-m] = (-1.0) ** l * np.conj(h)
            hJ = {}
            for mm in range(-l, l + 1):                 # first rotation, CP -> J
                acc = np.zeros(t.shape, dtype=np.complex128)
                for mp, h in cp.items():
                    acc += np.conj(paper_D(l, mm, mp, alpha, beta, gamma)) * h
                hJ[mm] = acc
            for mm in range(-l, l + 1):                 # second rotation, J -> L0
                acc = np.zeros(t.shape, dtype=np.complex128)
                for mp in range(-l, l + 1):
                    acc += np.conj(paper_D(l, mm, mp, *rot0)) * hJ[mp]
                hpc += acc * sYlm(-2, l, mm, iota, phr)
    hpc = hpc * np.exp(2j * src["psi"])
    return hpc.real, -hpc.imag
