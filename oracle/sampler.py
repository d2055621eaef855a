"""Fisher-Gaussian proposal and exact-likelihood Metropolis-Hastings step
(Sec. II.C, Fisher initialization; the sampler's accept rule).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. II.C draws starting points from a multivariate Gaussian whose mean is the
injection and whose covariance is the inverse Fisher matrix, the Fisher matrix
being built from finite differences of the likelihood.  Reading taken here:
F = -d^2 logL / dtheta dtheta at theta0 by central second differences of logL
(in zero noise at the injection this is (dh|dh)):
    F_aa = -(L(+a) - 2 L(0) + L(-a)) / eps_a^2
    F_ab = -(L(+a+b) - L(+a-b) - L(-a+b) + L(-a-b)) / (4 eps_a eps_b)
over the D sampled parameters idx.  The Gaussian q = N(mu, F^-1) is drawn as
x = mu + L^-T z with F = L L^T (z standard normal, passed in), so that
log q(x) = -|z|^2 / 2 + sum_i log L_ii - (D/2) log(2 pi), z = L^T (x - mu).
The Metropolis-Hastings step with an independence proposal accepts x' when
log u < [log pi(x') - log q(x')] - [log pi(x) - log q(x)], u uniform in (0, 1]
(passed in), pi = likelihood x uniform prior box (Table I's prior ranges);
a proposal outside the box or with logL = -inf is rejected.
"""
import math

import numpy as np
from scipy.linalg import solve_triangular


def n_fisher_points(D):
    return 1 + 2 * D + 2 * D * (D - 1)


def fisher_points(theta0, eps, idx):
    """Stencil points [P][15] in a fixed order: theta0; then per parameter a:
    +a, -a; then per pair a < b (lexicographic): ++, +-, -+, --."""
    theta0 = np.asarray(theta0, dtype=np.float64)
    D = len(idx)
    pts = [theta0.copy()]
    for a in range(D):
        for s in (1.0, -1.0):
            p = theta0.copy()
            p[idx[a]] += s * eps[a]
            pts.append(p)
    for a in range(D):
        for b in range(a + 1, D):
            for sa, sb in ((1.0, 1.0), (1.0, -1.0), (-1.0, 1.0), (-1.0, -1.0)):
                p = theta0.copy()
                p[idx[a]] += sa * eps[a]
                p[idx[b]] += sb * eps[b]
                pts.append(p)
    return np.array(pts)


def fisher_assemble(logl, eps, D):
    """F [D][D] from the logL values at ``fisher_points`` (same order)."""
    L0 = logl[0]
    F = np.zeros((D, D))
    for a in range(D):
        F[a, a] = -(logl[1 + 2 * a] - 2.0 * L0 + logl[2 + 2 * a]) / eps[a] ** 2
    k = 1 + 2 * D
    for a in range(D):
        for b in range(a + 1, D):
            pp, pm, mp, mm = logl[k:k + 4]
            F[a, b] = F[b, a] = -(pp - pm - mp + mm) / (4.0 * eps[a] * eps[b])
            k += 4
    return F


def cholesky(F):
    """Lower-triangular L with L L^T = F (library routine as one step)."""
    return np.linalg.cholesky(F)


def gauss_draw(mu, L, idx, z):
    """x = mu + L^-T z on the sampled parameters; -> (x [W][15], logq [W])."""
    z = np.atleast_2d(np.asarray(z, dtype=np.float64))
    D = len(idx)
    x = np.repeat(np.asarray(mu, dtype=np.float64)[None, :], z.shape[0], axis=0)
    y = solve_triangular(L.T, z.T, lower=False).T
    x[:, idx] += y
    logq = -0.5 * np.sum(z * z, axis=1) + np.sum(np.log(np.diag(L))) - 0.5 * D * math.log(2 * math.pi)
    return x, logq


def gauss_logq(mu, L, idx, x):
    """log q(x) of N(mu, (L L^T)^-1) on the sampled parameters."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    D = len(idx)
    dx = x[:, idx] - np.asarray(mu)[idx][None, :]
    z = dx @ L                      # rows: (L^T dx)^T
    return -0.5 * np.sum(z * z, axis=1) + np.sum(np.log(np.diag(L))) - 0.5 * D * math.log(2 * math.pi)


def gauss_walk(x, L, idx, z, step):
    """Random-walk proposal x' = x + step L^-T z on the sampled parameters
    (symmetric: log q terms cancel, pass log q = 0 to mh_accept)."""
    x = np.array(np.atleast_2d(x), dtype=np.float64)
    z = np.atleast_2d(np.asarray(z, dtype=np.float64))
    y = solve_triangular(L.T, z.T, lower=False).T
    x[:, idx] += step * y
    return x


def mh_accept(x, logl, logq, xp, loglp, logqp, u, lo, hi, beta=None):
    """One independence Metropolis-Hastings decision per walker (at inverse
    temperature beta[w], target pi^beta; beta = 1 when None).
    -> (x, logl, logq) after the step and the accepted flags (int)."""
    x = np.array(x, dtype=np.float64)
    logl = np.array(logl, dtype=np.float64)
    logq = np.array(logq, dtype=np.float64)
    acc = np.zeros(len(x), dtype=np.int32)
    for w in range(len(x)):
        inside = bool(np.all(xp[w] >= lo) and np.all(xp[w] <= hi))
        if not inside or not (loglp[w] > -math.inf):
            continue
        b = 1.0 if beta is None else beta[w]
        if math.log(u[w]) < (b * loglp[w] - logqp[w]) - (b * logl[w] - logq[w]):
            x[w] = xp[w]
            logl[w] = loglp[w]
            logq[w] = logqp[w]
            acc[w] = 1
    return x, logl, logq, acc


def pt_swap(x, logl, logq, betas, u):
    """Replica exchange between adjacent temperatures (ptemcee-style parallel
    tempering, the sampler of Sec. II.C): walkers are [T][W] (temperature
    major, beta decreasing with the index, beta[0] = 1); for k = T-2 down to 0
    the states of (k, w) and (k+1, w) are exchanged when
    log u[k][w] < (beta_k - beta_{k+1}) (logL_{k+1,w} - logL_{k,w}).
    x [T][W][15], logl / logq [T][W] are returned updated with the swap flags
    [T-1][W]; log q (of the proposal at each walker's position) moves with
    the state."""
    x = np.array(x, dtype=np.float64)
    logl = np.array(logl, dtype=np.float64)
    logq = np.array(logq, dtype=np.float64)
    T, W = logl.shape
    sw = np.zeros((T - 1, W), dtype=np.int32)
    for w in range(W):
        for k in range(T - 2, -1, -1):
            a = (betas[k] - betas[k + 1]) * (logl[k + 1, w] - logl[k, w])
            if math.log(u[k][w]) < a:
                x[[k, k + 1], w] = x[[k + 1, k], w]
                logl[[k, k + 1], w] = logl[[k + 1, k], w]
                logq[[k, k + 1], w] = logq[[k + 1, k], w]
                sw[k, w] = 1
    return x, logl, logq, sw
