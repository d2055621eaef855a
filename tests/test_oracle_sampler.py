"""Pins of the oracle's Fisher-Gaussian proposal and Metropolis-Hastings step
(Sec. II.C) against closed forms, a library density and the stationary
distribution of the chain -- nothing here re-types the oracle's formulas."""
import math

import numpy as np
from scipy.stats import multivariate_normal

from oracle import likelihood, pipeline, sampler
from paper_2501_08261_gb300 import workloads

from helpers import oracle_setup


def _spd(D, seed):
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(D, D))
    return Q @ Q.T + D * np.eye(D)


def test_fisher_is_exact_on_a_quadratic_loglike():
    # central second differences are exact on a quadratic: F must equal its Hessian
    D = 15
    A = _spd(D, 1)
    rng = np.random.default_rng(2)
    theta0 = rng.normal(size=15)
    idx = list(rng.permutation(15))
    eps = rng.uniform(1e-3, 1e-1, D)
    pts = sampler.fisher_points(theta0, eps, idx)
    assert pts.shape == (sampler.n_fisher_points(D), 15) == (451, 15)
    dx = pts[:, idx] - theta0[idx]
    logl = -0.5 * np.einsum("pi,ij,pj->p", dx, A, dx) + 3.7
    F = sampler.fisher_assemble(logl, eps, D)
    assert np.max(np.abs(F - A)) <= 1e-8 * np.max(np.abs(A))


def test_fisher_stencil_points_differ_from_theta0_in_at_most_two_entries():
    theta0 = np.arange(15.0)
    pts = sampler.fisher_points(theta0, [0.5, 0.25, 2.0], [3, 7, 11])
    nz = (pts != theta0).sum(axis=1)
    assert nz[0] == 0 and np.all(nz[1:7] == 1) and np.all(nz[7:] == 2)
    assert len(pts) == 1 + 2 * 3 + 4 * 3


def test_fisher_from_loglike_equals_dh_inner_product():
    # zero noise at the injection: -d^2 logL = (dh_a | dh_b)
    cfg = workloads.config("c1_fp64_1d")
    s = oracle_setup(cfg)
    theta = workloads.c1_point()
    d0 = pipeline.aet(theta, s)
    rho = math.sqrt(-2.0 * likelihood.loglike(np.zeros_like(d0), d0, s.dt, s.f_lo, s.f_hi, s.tdi_gen))
    theta[8] *= rho / 500.0                       # SNR 500
    d = pipeline.aet(theta, s)
    idx = [14, 8]
    eps = np.array([0.05, 1e-3 * theta[8]])
    pts = sampler.fisher_points(theta, eps, idx)
    logl = np.array([pipeline.loglike(p, s, d) for p in pts])
    F = sampler.fisher_assemble(logl, eps, 2)
    der = []
    for a in range(2):
        tp, tm = theta.copy(), theta.copy()
        tp[idx[a]] += eps[a]
        tm[idx[a]] -= eps[a]
        der.append((pipeline.aet(tp, s) - pipeline.aet(tm, s)) / (2 * eps[a]))
    f = likelihood.freqs(s.n, s.dt)
    mask = likelihood.band(s.n, s.dt, s.f_lo, s.f_hi)
    sae, st = likelihood.psd_aet(np.where(f > 0, f, 1.0), s.tdi_gen)
    df = 1.0 / (s.n * s.dt)
    G = np.zeros((2, 2))
    for a in range(2):
        for b in range(2):
            G[a, b] = sum(likelihood.inner(likelihood.dft(der[a][c], s.dt),
                                           likelihood.dft(der[b][c], s.dt),
                                           st if c == 2 else sae, df, mask) for c in range(3))
    assert np.all(np.abs(F - G) <= 2e-3 * np.sqrt(np.outer(np.diag(G), np.diag(G))))
    assert G[0, 0] > 0 and G[1, 1] > 0


def test_gauss_draw_density_and_covariance():
    D = 6
    F = _spd(D, 3)
    L = sampler.cholesky(F)
    assert np.allclose(L @ L.T, F, rtol=0, atol=1e-12 * np.max(F))
    mu = np.linspace(-1.0, 1.0, 15)
    idx = [0, 2, 5, 9, 13, 14]
    z = workloads.standard_normals(40000, D, 4)
    x, logq = sampler.gauss_draw(mu, L, idx, z)
    cov = np.linalg.inv(F)
    want = multivariate_normal(mean=mu[idx], cov=cov).logpdf(x[:, idx])
    assert np.max(np.abs(logq - want)) <= 1e-9 * np.max(np.abs(want))
    assert np.max(np.abs(sampler.gauss_logq(mu, L, idx, x) - logq)) <= 1e-10 * np.max(np.abs(logq))
    others = [k for k in range(15) if k not in idx]
    assert np.all(x[:, others] == mu[others])
    emp = np.cov((x[:, idx] - mu[idx]).T)
    assert np.max(np.abs(emp - cov)) <= 0.05 * np.max(np.abs(cov))


def test_mh_chain_has_the_target_as_stationary_distribution():
    # target N(1, 0.5^2) on parameter 0, independence proposal N(0, 1.5^2)
    W, steps = 256, 600
    rng = np.random.default_rng(5)
    mu = np.zeros(15)
    L = np.array([[1.0 / 1.5]])
    lo, hi = np.full(15, -10.0), np.full(15, 10.0)

    def logl_of(x):
        return -0.5 * ((x[:, 0] - 1.0) / 0.5) ** 2

    x, logq = sampler.gauss_draw(mu, L, [0], rng.normal(size=(W, 1)))
    logl = logl_of(x)
    keep = []
    for it in range(steps):
        xp, logqp = sampler.gauss_draw(mu, L, [0], rng.normal(size=(W, 1)))
        x, logl, logq, acc = sampler.mh_accept(x, logl, logq, xp, logl_of(xp), logqp,
                                               rng.uniform(1e-300, 1.0, W), lo, hi)
        if it >= 100:
            keep.append(x[:, 0].copy())
    s = np.concatenate(keep)
    assert abs(s.mean() - 1.0) < 0.02
    assert abs(s.std() - 0.5) < 0.02


def test_mh_rejects_outside_box_and_minus_infinity():
    W = 8
    x = np.zeros((W, 15))
    logl = np.full(W, -5.0)
    logl[7] = -math.inf                              # a walker that starts invalid
    logq = np.zeros(W)
    xp = np.full((W, 15), 0.5)
    xp[0, 3] = 2.0                                  # outside the box
    loglp = np.full(W, 10.0)
    loglp[1] = -math.inf
    lo, hi = np.full(15, -1.0), np.full(15, 1.0)
    u = np.full(W, 0.999)
    xn, ln, qn, acc = sampler.mh_accept(x, logl, logq, xp, loglp, np.zeros(W), u, lo, hi)
    assert acc[0] == 0 and acc[1] == 0 and np.all(acc[2:] == 1)
    assert np.all(xn[0] == 0.0) and ln[1] == -5.0 and ln[7] == 10.0


def test_random_walk_chain_targets_a_correlated_gaussian():
    # target N(0, C) in 2-d through the Fisher factor of C^-1: stationary moments
    C = np.array([[1.0, 0.8], [0.8, 1.0]])
    L = sampler.cholesky(np.linalg.inv(C))
    rng = np.random.default_rng(8)
    W, idx = 256, [2, 9]
    lo, hi = np.full(15, -50.0), np.full(15, 50.0)
    Ci = np.linalg.inv(C)

    def logl_of(x):
        y = x[:, idx]
        return -0.5 * np.einsum("wi,ij,wj->w", y, Ci, y)

    x = np.zeros((W, 15))
    logl, zero = logl_of(x), np.zeros(W)
    keep = []
    for it in range(800):
        xp = sampler.gauss_walk(x, L, idx, rng.normal(size=(W, 2)), 2.38 / np.sqrt(2))
        x, logl, _, _ = sampler.mh_accept(x, logl, zero, xp, logl_of(xp), zero,
                                          rng.uniform(1e-300, 1.0, W), lo, hi)
        if it >= 200:
            keep.append(x[:, idx].copy())
    s = np.concatenate(keep)
    assert np.allclose(np.cov(s.T), C, atol=0.06)
    assert np.all(np.abs(s.mean(axis=0)) < 0.05)


def test_tempered_chains_and_swaps_target_the_tempered_posteriors():
    # target N(0, 1) on parameter 0; at inverse temperature b the chain samples
    # N(0, 1/b), whatever the swaps between temperatures do
    betas = np.array([1.0, 0.5, 0.25])
    T, W = 3, 128
    rng = np.random.default_rng(9)
    mu = np.zeros(15)
    L = np.array([[1.0 / 2.5]])                       # proposal N(0, 2.5^2)
    lo, hi = np.full(15, -40.0), np.full(15, 40.0)
    beta_w = np.repeat(betas, W)

    def logl_of(x):
        return -0.5 * x[:, 0] ** 2

    x, logq = sampler.gauss_draw(mu, L, [0], rng.normal(size=(T * W, 1)))
    logl = logl_of(x)
    keep = [[] for _ in range(T)]
    nsw = 0
    for it in range(700):
        xp, logqp = sampler.gauss_draw(mu, L, [0], rng.normal(size=(T * W, 1)))
        x, logl, logq, _ = sampler.mh_accept(x, logl, logq, xp, logl_of(xp), logqp,
                                             rng.uniform(1e-300, 1.0, T * W), lo, hi, beta_w)
        xs, ls, qs, sw = sampler.pt_swap(x.reshape(T, W, 15), logl.reshape(T, W),
                                         logq.reshape(T, W), betas,
                                         rng.uniform(1e-300, 1.0, (T - 1, W)))
        x, logl, logq = xs.reshape(T * W, 15), ls.ravel(), qs.ravel()
        nsw += sw.sum()
        if it >= 100:
            for k in range(T):
                keep[k].append(xs[k, :, 0].copy())
    for k in range(T):
        v = np.concatenate(keep[k]).var()
        assert abs(v * betas[k] - 1.0) < 0.06, (k, v)
    assert nsw > 0
