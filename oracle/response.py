"""Time-domain LISA response (Sec. II.B): link responses y_slr (Eq. yslr),
TDI Michelson X 1.5 / 2.0, Y and Z by cyclic permutation, and A, E, T.

Readings of the paper taken here:
* h at the off-grid times t_s, t_r and y at the delayed TDI times come from
  centred Lagrange interpolation of order p (odd; p = 1 is the paper's linear
  interpolation, Sec. II.B end); samples outside the grid are zero.
* y_slr = [x+ dh+ + 2 x_x dh_x] / (2 (1 - k.n)), i.e. n_i n_j h_ij / 2 with
  e_x = u(x)v + v(x)u; positions in light-seconds; sender at t - L_l(t).
* every TDI delay is the plain sum of the light times evaluated at the
  output time t (the printed form); with ``nested=True`` each term's delay is
  instead the product of one-link delay operators, applied from the output
  time backwards (the chains below).
* the third y_123 term of X_2 carries the delay 2L_-2 + L_2 + 2L_3 + 2L_-3.
"""
import math

import numpy as np

from . import orbits

# X_1.5 as printed: (link, sign, links whose light times sum to the delay);
# y_{1-32} is link -3, y_{231} link 3, y_{123} link 2, y_{3-21} link -2.
X15_TERMS = (
    (-3, +1, (3, 2, -2)), (-3, -1, (3,)),
    (3, +1, (2, -2)), (3, -1, ()),
    (2, +1, (-2,)), (2, -1, (-2, -3, 3)),
    (-2, +1, ()), (-2, -1, (-3, 3)),
)
# X_2 as printed, with the y_123 third-term delay read as 2L-2 + L2 + 2L3 + 2L-3
X20_TERMS = (
    (-3, +1, (3, 2, -2)), (-3, -1, (3,)),
    (-3, +1, (-2, 2, 3, 3, -3)), (-3, -1, (3, 3, -3, -2, -2, 2, 2)),
    (3, +1, (2, -2)), (3, -1, ()),
    (3, +1, (-2, 2, 3, -3)), (3, -1, (3, -3, -2, -2, 2, 2)),
    (2, +1, (-2,)), (2, -1, (-2, -3, 3)),
    (2, +1, (-2, -2, 2, 3, 3, -3, -3)), (2, -1, (3, -3, -2, -2, 2)),
    (-2, +1, ()), (-2, -1, (-3, 3)),
    (-2, +1, (-2, 2, 3, 3, -3, -3)), (-2, -1, (3, -3, -2, 2)),
)


# The same terms with each delay as a product of one-link operators,
# D_a f(t) = f(t - L_a(t)), the first link of a chain applied at the output
# time and each next one at the output time minus the delay so far.  Writing
# D_ijk.. for the path received at i from j, at j from k, ..., X factors as
#   X_1.5 = (1 - D_121)(y_{3-21} + D_13 y_123) - (1 - D_131)(y_231 + D_12 y_{1-32})
#   X_2   = (1 - D_121 - D_12131 + D_1312121)(y_{3-21} + D_13 y_123)
#         - (1 - D_131 - D_13121 + D_1213131)(y_231 + D_12 y_{1-32}),
# and every printed term is exactly one product of that expansion (same link,
# sign and multiset of light times).  D_12 is link 3, D_21 link -3, D_13
# link -2, D_31 link 2.  Order and entries follow X15_TERMS / X20_TERMS.
X15_CHAINS = (
    (-3, +1, (-2, 2, 3)), (-3, -1, (3,)),
    (3, +1, (-2, 2)), (3, -1, ()),
    (2, +1, (-2,)), (2, -1, (3, -3, -2)),
    (-2, +1, ()), (-2, -1, (3, -3)),
)
X20_CHAINS = (
    (-3, +1, (-2, 2, 3)), (-3, -1, (3,)),
    (-3, +1, (-2, 2, 3, -3, 3)), (-3, -1, (3, -3, -2, 2, -2, 2, 3)),
    (3, +1, (-2, 2)), (3, -1, ()),
    (3, +1, (-2, 2, 3, -3)), (3, -1, (3, -3, -2, 2, -2, 2)),
    (2, +1, (-2,)), (2, -1, (3, -3, -2)),
    (2, +1, (-2, 2, 3, -3, 3, -3, -2)), (2, -1, (3, -3, -2, 2, -2)),
    (-2, +1, ()), (-2, -1, (3, -3)),
    (-2, +1, (-2, 2, 3, -3, 3, -3)), (-2, -1, (3, -3, -2, 2)),
)


def cyclic(link, times=1):
    """Index permutation 1 -> 2 -> 3 -> 1 on |l|, sign kept (Y: once, Z: twice)."""
    a = abs(link)
    for _ in range(times):
        a = a % 3 + 1
    return a if link > 0 else -a


def channel_terms(gen, channel, nested=False):
    """Terms of X (channel 0), Y (1) or Z (2) for TDI generation 15 or 20
    (delay links in operator order when ``nested``)."""
    if nested:
        base = X15_CHAINS if gen == 15 else X20_CHAINS
    else:
        base = X15_TERMS if gen == 15 else X20_TERMS
    return [(cyclic(l, channel), sg, tuple(cyclic(d, channel) for d in dl))
            for (l, sg, dl) in base]


# ---------------------------------------------------------------------------
# Lagrange interpolation
# ---------------------------------------------------------------------------

def lagrange_offsets(p):
    """Node offsets -(p-1)/2 .. (p+1)/2 of the centred order-p stencil."""
    if p < 1 or p % 2 == 0:
        raise ValueError("Lagrange order must be odd")
    return np.arange(p + 1) - (p - 1) // 2


def lagrange_weights(eps, p):
    """w_j(eps) = prod_{m != j} (eps - o_m)/(o_j - o_m), shape eps.shape + (p+1,)."""
    o = lagrange_offsets(p).astype(np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    d = eps[..., None] - o                           # eps - o_m
    ones = np.ones(eps.shape + (1,))
    pre = np.cumprod(np.concatenate([ones, d[..., :-1]], axis=-1), axis=-1)
    suf = np.cumprod(np.concatenate([ones, d[..., :0:-1]], axis=-1), axis=-1)[..., ::-1]
    denom = np.array([np.prod([o[j] - o[m] for m in range(p + 1) if m != j])
                      for j in range(p + 1)])
    return pre * suf / denom


def interp(series, tau, p):
    """series evaluated at fractional sample positions tau (zero outside)."""
    tau = np.asarray(tau, dtype=np.float64)
    out = np.zeros(tau.shape)
    step = 1 << 16
    flat_t = tau.reshape(-1)
    flat_o = out.reshape(-1)
    o = lagrange_offsets(p)
    n = series.shape[0]
    for a in range(0, flat_t.size, step):
        tt = flat_t[a:a + step]
        i = np.floor(tt)
        w = lagrange_weights(tt - i, p)
        idx = i.astype(np.int64)[:, None] + o
        ok = (idx >= 0) & (idx < n)
        vals = np.where(ok, series[np.clip(idx, 0, n - 1)], 0.0)
        flat_o[a:a + step] = np.sum(w * vals, axis=-1)
    return out


# ---------------------------------------------------------------------------
# link response, Eq. (yslr)
# ---------------------------------------------------------------------------

def source_basis(beta, lam):
    """Propagation vector k and polarisation vectors u, v (Sec. II.B)."""
    cb, sb, cl, sl = math.cos(beta), math.sin(beta), math.cos(lam), math.sin(lam)
    k = np.array([-cb * cl, -cb * sl, -sb])
    v = np.array([-sb * cl, -sb * sl, cb])
    u = np.array([sl, -cl, 0.0])
    return k, u, v


def link_response(hp, hc, t0, dt, orbit, link, beta, lam, idx, p):
    """y_slr at grid indices idx for link (s, l, r) from h+, hx on the grid."""
    k, u, v = source_basis(beta, lam)
    t = t0 + np.asarray(idx, dtype=np.float64) * dt
    rr, rs, n, L = orbits.link_geometry(orbit, link, t)
    ts = t - L - rs @ k
    tr = t - rr @ k
    un, vn, kn = n @ u, n @ v, n @ k
    xp = un * un - vn * vn
    xc = un * vn
    dhp = interp(hp, (ts - t0) / dt, p) - interp(hp, (tr - t0) / dt, p)
    dhc = interp(hc, (ts - t0) / dt, p) - interp(hc, (tr - t0) / dt, p)
    return (xp * dhp + 2.0 * xc * dhc) / (2.0 * (1.0 - kn))


def all_links(hp, hc, t0, dt, orbit, beta, lam, p, idx=None):
    """y for the six links (order orbits.LINKS) on the grid (or at idx)."""
    n = hp.shape[0]
    if idx is None:
        idx = np.arange(n)
    return {l: link_response(hp, hc, t0, dt, orbit, l, beta, lam, idx, p)
            for l in orbits.LINKS}


# ---------------------------------------------------------------------------
# TDI and A, E, T
# ---------------------------------------------------------------------------

def nested_delay(orbit, chain, t):
    """Delay of the operator product D_{c1} D_{c2} ... at output times t:
    tau = 0, then tau += L_c(t - tau) for each link c in operator order."""
    t = np.asarray(t, dtype=np.float64)
    tau = np.zeros(t.shape)
    for c in chain:
        tau = tau + orbits.light_time(orbit, c, t - tau)
    return tau


def term_delays(orbit, gen, channel, t, nested=False):
    """(link, sign, delay at t) of every term of one channel."""
    out = []
    if nested:
        for (link, sign, chain) in channel_terms(gen, channel, True):
            out.append((link, sign, nested_delay(orbit, chain, t)))
        return out
    L = {l: orbits.light_time(orbit, l, t) for l in orbits.LINKS}
    for (link, sign, delays) in channel_terms(gen, channel):
        D = np.zeros(np.shape(t))
        for d in delays:
            D = D + L[d]
        out.append((link, sign, D))
    return out


def tdi_xyz(y, n, t0, dt, orbit, gen, p, idx=None, nested=False):
    """X, Y, Z at grid indices idx (default all) from y[link] on the full grid."""
    if idx is None:
        idx = np.arange(n)
    idx = np.asarray(idx)
    t = t0 + idx.astype(np.float64) * dt
    out = []
    for ch in range(3):
        acc = np.zeros(idx.shape)
        for (link, sign, D) in term_delays(orbit, gen, ch, t, nested):
            acc = acc + sign * interp(y[link], idx - D / dt, p)
        out.append(acc)
    return out


def aet_from_xyz(X, Y, Z):
    """A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6, T = (X + Y + Z)/sqrt3."""
    return ((Z - X) / math.sqrt(2.0), (X - 2.0 * Y + Z) / math.sqrt(6.0),
            (X + Y + Z) / math.sqrt(3.0))


def tdi_support(idx, n, dt, orbit, gen, p, t0=0.0, nested=False):
    """Grid indices of y that the TDI outputs at idx read (for sparse runs)."""
    idx = np.asarray(idx)
    t = t0 + idx * dt
    o = lagrange_offsets(p)
    need = set()
    for ch in range(3):
        for (link, sign, D) in term_delays(orbit, gen, ch, t, nested):
            base = np.floor(idx - D / dt).astype(np.int64)
            for b in base:
                need.update((b + o).tolist())
    need = np.array(sorted(j for j in need if 0 <= j < n), dtype=np.int64)
    return need
