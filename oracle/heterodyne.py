"""Heterodyned time-domain likelihood (the paper names heterodyning and
relative binning as the route to cheaper likelihoods, Sec. I and Sec. IV,
and gives no time-domain form; the definition below is this library's).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Definition.  Grid t_i = t0 + i dt, i < n; fiducial parameters theta0; node
indices 0 = i_0 < i_1 < ... < i_{B-1} = n - 1.

1. Analytic mode polarisations.  The contribution of one mode pair
   j = (l, +-m) to h+ - i hx (after the psi rotation) is
       S_j = e^{2 i psi} (h_lm Y+ + (-1)^l conj(h_lm) Y-),
   with h_lm = A e^{-i Phi_lm} the aligned / co-precessing mode and Y+-
   its angular factors (-2Y_{l,+-m}(iota, phi_ref), or for precessing spins
   the two-step twist-up of a unit co-precessing mode +-m).  With
   P = e^{2 i psi} Y+, Q = e^{2 i psi} Y-, sg = (-1)^l:
       hp_j = h_lm (P + sg conj Q),   hx_j = i h_lm (P - sg conj Q),
   so Re hp_j and Re hx_j are the pair's h+ and hx, and both carry the single
   phase e^{-i Phi_lm}.  hp_j = hx_j = 0 outside [t0, t_{n-1}] (the sampled
   path's samples outside the grid are zero).
2. Complex channel response.  X_jc(t) is TDI channel c (A, E, T) of the link
   responses to (hp_j, hx_j), evaluated in continuous time: every term of
   X, Y, Z at output time t reads link l at t' = t - D(t) (D as in
   ``response.term_delays``), the link geometry at t', and the waveform at the
   exact emission and reception times t' - L - k.r_s and t' - k.r_r of
   Eq. (yslr) (no interpolation); a term whose t' leaves the grid reads 0.
   Re sum_j X_jc is the continuous-time A, E, T that the sampled path
   approximates with Lagrange interpolation.
3. Carriers.  C_j(t) = e^{-i Phi_lm(t; theta0)}, the fiducial's own mode phase.
4. Node differences.  dZ_jc,b = conj(C_j(t_b)) [X_jc(t_b; theta) - X_jc(t_b; theta0)]
   at the nodes t_b = t0 + i_b dt: slowly varying where theta is near theta0.
5. Model.  For i_b <= i < i_{b+1} (B >= 4 nodes), the cubic Lagrange polynomial
   through the four nodes a .. a + 3, a = min(max(b - 1, 0), B - 4) (the
   stencil moved inwards at the ends):
       h_c(t_i) = X0_c(t_i) + Re sum_j C_j(t_i) sum_q w_q(i) dZ_jc,a+q,
       w_q(i) = prod_{r != q} (i - i_{a+r}) / (i_{a+q} - i_{a+r}),
   X0_c = Re sum_j X_jc(t_i; theta0), the fiducial's continuous-time response
   on the grid.  At theta = theta0 every dZ is 0 and the model is X0; with a
   node at every sample it is Re sum_j X_jc(t_i; theta), the continuous-time
   response of theta itself (``continuous_aet``).
6. logL = ``likelihood.loglike`` of the model against the data (same DFT,
   PSD, band and channels as the full likelihood).

The heterodyned likelihood therefore approximates the likelihood of the
continuous-time response, of which the sampled path (Lagrange interpolation
of h on the grid, then of y) is the paper's discretisation.  The two agree to
the interpolation error of the sampled path: ~1e-13 of the signal where h is
band-limited, but up to ~1e-4 within a few stencil widths of the stand-in's
merger attachment, where h is only C1 (its second derivative jumps at t_m).
"""

import numpy as np

from . import likelihood, orbits, pipeline, response, waveform
from .wigner import sYlm


def _angular(src, l, m, t, precessing):
    """Angular factors (Y+, Y-) of the co-precessing / aligned pair (l, +-m)
    at times t, before the psi rotation."""
    iota, phr = src["iota"], src["phi_ref"]
    if not precessing:
        one = np.ones(np.shape(t))
        return sYlm(-2, l, m, iota, phr) * one, sYlm(-2, l, -m, iota, phr) * one
    alpha, beta, gamma, rot0 = waveform.euler_angles(src, t)
    out = []
    for mp in (m, -m):
        # a unit co-precessing mode mp through CP -> J -> L0, then onto -2Y_l
        hJ = {mq: np.conj(waveform.paper_D(l, mq, mp, alpha, beta, gamma))
              for mq in range(-l, l + 1)}
        acc = np.zeros(np.shape(t), dtype=np.complex128)
        for mm in range(-l, l + 1):
            hL = np.zeros(np.shape(t), dtype=np.complex128)
            for mq in range(-l, l + 1):
                hL = hL + np.conj(waveform.paper_D(l, mm, mq, *rot0)) * hJ[mq]
            acc = acc + hL * sYlm(-2, l, mm, iota, phr)
        out.append(acc)
    return out[0], out[1]


def analytic_modes(theta, t, s: pipeline.Setup):
    """[(l, m, hp_j, hx_j)] at times t (step 1), zero outside the grid."""
    src = waveform.source(theta, s.precessing)
    t = np.asarray(t, dtype=np.float64)
    t_end = s.t0 + (s.n - 1) * s.dt
    inside = (t >= s.t0) & (t <= t_end)
    rot = np.exp(2j * src["psi"])
    out = []
    for (l, m) in waveform.modes_from_mask(s.mode_mask):
        h = np.where(inside, waveform.mode(src, l, m, t, s.t0), 0.0)
        yp, ym = _angular(src, l, m, t, s.precessing)
        P, Q = rot * yp, rot * ym
        sg = (-1.0) ** l
        out.append((l, m, h * (P + sg * np.conj(Q)), 1j * h * (P - sg * np.conj(Q))))
    return out


def point_aet(theta, s: pipeline.Setup, t_out):
    """X_jc at output times t_out (step 2): complex [n_modes][3][len(t_out)]."""
    t_out = np.asarray(t_out, dtype=np.float64)
    k, u, v = response.source_basis(theta[11], theta[12])
    t_end = s.t0 + (s.n - 1) * s.dt
    nm = len(waveform.modes_from_mask(s.mode_mask))
    xyz = np.zeros((nm, 3, t_out.size), dtype=np.complex128)
    for ch in range(3):
        for (link, sign, D) in response.term_delays(s.orbit, s.tdi_gen, ch, t_out,
                                                    s.tdi_nested):
            tp = t_out - D
            inside = (tp >= s.t0) & (tp <= t_end)
            rr, rs, n, L = orbits.link_geometry(s.orbit, link, tp)
            ts = tp - L - rs @ k
            tr = tp - rr @ k
            un, vn, kn = n @ u, n @ v, n @ k
            xp = un * un - vn * vn
            xc = un * vn
            at_s = analytic_modes(theta, ts, s)
            at_r = analytic_modes(theta, tr, s)
            for j in range(nm):
                y = (xp * (at_s[j][2] - at_r[j][2]) + 2.0 * xc * (at_s[j][3] - at_r[j][3])) \
                    / (2.0 * (1.0 - kn))
                xyz[j, ch] += sign * np.where(inside, y, 0.0)
    A, E, T = response.aet_from_xyz(xyz[:, 0], xyz[:, 1], xyz[:, 2])
    return np.stack([A, E, T], axis=1)


def carriers(theta0, s: pipeline.Setup, t):
    """C_j(t) = e^{-i Phi_lm(t; theta0)} (step 3): complex [n_modes][len(t)]."""
    src = waveform.source(theta0, s.precessing)
    return np.stack([np.exp(-1j * waveform.mode_phase(src, l, m, t)[0])
                     for (l, m) in waveform.modes_from_mask(s.mode_mask)])


def node_deltas(theta, theta0, s: pipeline.Setup, node_idx):
    """dZ_jc,b (step 4): complex [n_modes][3][B]."""
    tb = s.t0 + np.asarray(node_idx, dtype=np.float64) * s.dt
    c = carriers(theta0, s, tb)
    return np.conj(c)[:, None, :] * (point_aet(theta, s, tb) - point_aet(theta0, s, tb))


def expand(dz, theta0, s: pipeline.Setup, node_idx, x0):
    """The model A, E, T on the grid (step 5) from node differences dz."""
    node_idx = np.asarray(node_idx, dtype=np.int64)
    B = node_idx.size
    if B < 4 or node_idx[0] != 0 or node_idx[-1] != s.n - 1 or np.any(np.diff(node_idx) <= 0):
        raise ValueError("nodes must be at least four, rising strictly from 0 to n - 1")
    i = np.arange(s.n)
    b = np.clip(np.searchsorted(node_idx, i, side="right") - 1, 0, B - 2)
    a = np.clip(b - 1, 0, B - 4)
    x = node_idx[a[:, None] + np.arange(4)].astype(np.float64)      # [n][4]
    w = np.ones((s.n, 4))
    for q in range(4):
        for r in range(4):
            if r != q:
                w[:, q] *= (i - x[:, r]) / (x[:, q] - x[:, r])
    c = carriers(theta0, s, pipeline.grid(s))
    out = np.array(x0, dtype=np.float64, copy=True)
    for j in range(dz.shape[0]):
        for ch in range(3):
            env = sum(w[:, q] * dz[j, ch, a + q] for q in range(4))
            out[ch] += (c[j] * env).real
    return out


def continuous_aet(theta, s: pipeline.Setup):
    """Re sum_j X_jc on the whole grid: the continuous-time A, E, T."""
    return point_aet(theta, s, pipeline.grid(s)).sum(axis=0).real


def model_aet(theta, theta0, s: pipeline.Setup, node_idx, x0=None):
    if x0 is None:
        x0 = continuous_aet(theta0, s)
    return expand(node_deltas(theta, theta0, s, node_idx), theta0, s, node_idx, x0)


def loglike(theta, theta0, s: pipeline.Setup, data_aet, node_idx, x0=None):
    """Step 6: -1/2 sum_c (h_c - d_c | h_c - d_c) with the heterodyned h."""
    h = model_aet(theta, theta0, s, node_idx, x0)
    return likelihood.loglike(h, data_aet, s.dt, s.f_lo, s.f_hi, s.tdi_gen, s.channel_mask)
