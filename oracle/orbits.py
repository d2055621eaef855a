"""Spacecraft orbits and link light times (Sec. II.B: the response needs both
ends' positions and every link's light time at each time of the observation).

Positions are in light-seconds in an ecliptic SSB frame.  Two declared models:

* ``rigid``  (equal-arm, stand-in for LDC's AnalyticOrbit): an equilateral
  triangle of side L with its centre on a 1 AU circle, its plane tilted 60 deg
  to the ecliptic, cartwheeling at -Omega.  Light time of every link = L/c.
* ``kepler`` (unequal-arm stand-in for the ESA file): each spacecraft on its own
  heliocentric Kepler ellipse (a = 1 AU, e_k = e0 (1 + eta_k), inclination
  i_k = sqrt(3) e_k, node turned by 2 pi (k-1)/3).  Light times solve
  |r_r(t) - r_s(t - L)| = L (light-seconds) by fixed-point iteration.

Link convention (Sec. II.B; y_slr labelled as in the TDI reference it cites):
link l is the arm opposite spacecraft |l|; +l and -l are its two directions.
"""
import math

import numpy as np

from . import consts as K

# l -> (sender, receiver); read off the y_slr labels of the X_1.5 equation
# (y_{1-32}, y_{231}, y_{123}, y_{3-21}) and completed by cyclic permutation.
LINK_ENDS = {1: (3, 2), 2: (1, 3), 3: (2, 1), -1: (2, 3), -2: (3, 1), -3: (1, 2)}
LINKS = (1, 2, 3, -1, -2, -3)            # storage order of the six links


def _guiding_frame(t):
    """Radial, azimuthal and vertical unit vectors of the 1 AU guiding centre."""
    a = K.OMEGA_ORB * np.asarray(t, dtype=np.float64)
    er = np.stack([np.cos(a), np.sin(a), np.zeros_like(a)], axis=-1)
    ephi = np.stack([-np.sin(a), np.cos(a), np.zeros_like(a)], axis=-1)
    ez = np.zeros_like(er)
    ez[..., 2] = 1.0
    return er, ephi, ez


def rigid_position(craft, t):
    """Position [.., 3] of spacecraft ``craft`` (1..3) at times t, rigid model.

    r_k = R_c + (L/sqrt3) [ -cos(Omega t - Th_k) u_hat + sin(Omega t - Th_k) e_phi ]
    with u_hat = (e_r + sqrt3 e_z)/2 and Th_k = 2 pi (k-1)/3.
    """
    t = np.asarray(t, dtype=np.float64)
    er, ephi, ez = _guiding_frame(t)
    centre = K.AU_S * er
    uhat = 0.5 * er + 0.5 * math.sqrt(3.0) * ez
    ang = K.OMEGA_ORB * t - 2.0 * math.pi * (craft - 1) / 3.0
    rho = K.ARM_S / math.sqrt(3.0)
    return centre + rho * (-np.cos(ang)[..., None] * uhat + np.sin(ang)[..., None] * ephi)


def _solve_kepler(mean_anom, e):
    """Eccentric anomaly E with E - e sin E = M (Newton to convergence)."""
    E = np.array(mean_anom, dtype=np.float64, copy=True)
    for _ in range(50):
        dE = (E - e * np.sin(E) - mean_anom) / (1.0 - e * np.cos(E))
        E = E - dE
        if np.max(np.abs(dE)) < 1e-15:
            break
    return E


def kepler_position(craft, t):
    """Position [.., 3] of spacecraft ``craft`` at times t, Keplerian model."""
    t = np.asarray(t, dtype=np.float64)
    e = K.KEPLER_E0 * (1.0 + K.KEPLER_ETA[craft - 1])
    inc = math.sqrt(3.0) * e
    node = 2.0 * math.pi * (craft - 1) / 3.0
    E = _solve_kepler(K.OMEGA_ORB * t - node, e)
    X = K.AU_S * (np.cos(E) - e)
    Y = K.AU_S * math.sqrt(1.0 - e * e) * np.sin(E)
    xt, zt = X * math.cos(inc), -X * math.sin(inc)
    x = xt * math.cos(node) - Y * math.sin(node)
    y = xt * math.sin(node) + Y * math.cos(node)
    return np.stack([x, y, zt], axis=-1)


class OrbitTable:
    """Spacecraft positions given as a table, the form of a mission orbit file
    (Sec. II.B needs the positions at every time of the observation; Sec. III.C
    runs on such a file).  Row j holds the three spacecraft's positions [m] at
    time t0 + j dt; pos_m has shape [rows][3][3] (row, spacecraft 1..3, x y z).

    Positions at other times (declared reading: the paper does not say how it
    resamples its orbit file): the degree-7 Lagrange polynomial through the
    eight rows j - 3 .. j + 4 around j = floor((t - t0) / dt), the eight rows
    moved inwards where they would leave the table."""

    def __init__(self, t0, dt, pos_m):
        self.t0 = float(t0)
        self.dt = float(dt)
        self.pos = np.asarray(pos_m, dtype=np.float64) / K.C_SI   # light-seconds
        if self.pos.ndim != 3 or self.pos.shape[1:] != (3, 3) or self.pos.shape[0] < 8:
            raise ValueError("orbit table must be [rows >= 8][3][3]")

    def position(self, craft, t):
        t = np.asarray(t, dtype=np.float64)
        x = (t - self.t0) / self.dt
        rows = self.pos.shape[0]
        first = np.clip(np.floor(x).astype(np.int64) - 3, 0, rows - 8)
        u = x - first                                   # in units of rows, nodes 0..7
        out = np.zeros(t.shape + (3,))
        for k in range(8):
            w = np.ones_like(u)
            for m in range(8):
                if m != k:
                    w = w * (u - m) / (k - m)
            out = out + w[..., None] * self.pos[first + k, craft - 1, :]
        return out


def position(kind, craft, t):
    """Position of ``craft`` at times t for orbit model ``kind``.

    Besides "rigid" and "kepler", two frozen constellations serve the closed-form
    pins: "static_rigid" (the rigid triangle at t = 0, equal arms) and
    "static_kepler" (the Keplerian positions at t = 0, unequal arms); an
    ``OrbitTable`` gives the caller's positions."""
    if isinstance(kind, OrbitTable):
        return kind.position(craft, t)
    if kind == "rigid":
        return rigid_position(craft, t)
    if kind == "kepler":
        return kepler_position(craft, t)
    t = np.asarray(t, dtype=np.float64)
    if kind == "static_rigid":
        return np.broadcast_to(rigid_position(craft, 0.0), t.shape + (3,))
    if kind == "static_kepler":
        return np.broadcast_to(kepler_position(craft, 0.0), t.shape + (3,))
    raise ValueError(kind)


def light_time(kind, link, t, iters=8):
    """Light travel time L_l(t) [s] of link ``link`` for reception at time t."""
    t = np.asarray(t, dtype=np.float64)
    if isinstance(kind, str) and kind in ("rigid", "static_rigid"):
        return np.full(t.shape, K.ARM_S)
    s, r = LINK_ENDS[link]
    if isinstance(kind, str) and kind == "static_kepler":
        return np.full(t.shape, float(np.linalg.norm(position(kind, r, 0.0)
                                                     - position(kind, s, 0.0))))
    rr = position(kind, r, t)
    L = np.linalg.norm(rr - position(kind, s, t), axis=-1)
    for _ in range(iters):
        L = np.linalg.norm(rr - position(kind, s, t - L), axis=-1)
    return L


def link_geometry(kind, link, t):
    """Receiver position r_r(t), emission position r_s(t - L_l), unit vector n,
    and light time L_l, all at reception times t (Eq. yslr)."""
    s, r = LINK_ENDS[link]
    L = light_time(kind, link, t)
    rr = position(kind, r, t)
    rs = position(kind, s, np.asarray(t, dtype=np.float64) - L)
    d = rr - rs
    n = d / np.linalg.norm(d, axis=-1, keepdims=True)
    return rr, rs, n, L
