"""Parity of the GPU proposal / accept kernels (include/lisa_sampler.h) with the
oracle's (oracle/sampler.py) on the same inputs, through the C ABI."""
import math

import numpy as np
import pytest

from oracle import pipeline, sampler
from paper_2501_08261_gb300 import api, workloads

from helpers import gpu_kwargs, oracle_setup

pytestmark = [pytest.mark.gpu]
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2501_08261_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _spd(D, seed):
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(D, D))
    return Q @ Q.T + D * np.eye(D)


@pytest.mark.parametrize("D", [1, 2, 7, 15])
def test_fisher_points_and_assemble_match_oracle(D):
    rng = np.random.default_rng(10 + D)
    theta0 = rng.normal(size=15) * 10.0
    idx = list(rng.permutation(15)[:D])
    eps = rng.uniform(1e-3, 1.0, D)
    P = api.lisa_fisher_npoints(D)
    pts = torch.empty((P, 15), dtype=torch.float64, device="cuda")
    api.lisa_fisher_points(_t(theta0), idx, eps, pts)
    want = sampler.fisher_points(theta0, eps, idx)
    assert np.array_equal(pts.cpu().numpy(), want)            # same additions: bit-exact
    logl = rng.normal(size=P) * 100.0 - 1e3
    F = torch.empty((D, D), dtype=torch.float64, device="cuda")
    api.lisa_fisher_assemble(_t(logl), eps, F)
    Fo = sampler.fisher_assemble(logl, eps, D)
    assert np.max(np.abs(F.cpu().numpy() - Fo)) <= 1e-15 * np.max(np.abs(Fo))


def test_cholesky_matches_library_and_flags_indefinite():
    for D in (1, 5, 15):
        A = _spd(D, D)
        L = torch.empty((D, D), dtype=torch.float64, device="cuda")
        info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        api.lisa_cholesky(_t(A), D, L, info)
        Lg = L.cpu().numpy()
        assert info.item() == 0
        assert np.max(np.abs(Lg - sampler.cholesky(A))) <= 1e-13 * np.max(np.abs(Lg))
        assert np.all(np.triu(Lg, 1) == 0.0)
    # a diagonal added before factorising (prior precision)
    A = _spd(6, 11)
    dg = np.linspace(0.5, 3.0, 6)
    L = torch.empty((6, 6), dtype=torch.float64, device="cuda")
    info = torch.zeros((1,), dtype=torch.int32, device="cuda")
    api.lisa_cholesky(_t(A), 6, L, info, diag=dg)
    assert info.item() == 0
    assert np.max(np.abs(L.cpu().numpy() - sampler.cholesky(A + np.diag(dg)))) <= 1e-13 * np.max(np.abs(A))
    B = _spd(4, 9)
    B[2, 2] = -1.0
    L = torch.empty((4, 4), dtype=torch.float64, device="cuda")
    info = torch.zeros((1,), dtype=torch.int32, device="cuda")
    api.lisa_cholesky(_t(B), 4, L, info)
    assert info.item() == 3


def test_gauss_draw_and_logq_match_oracle():
    D, W = 9, 1000
    F = _spd(D, 21)
    L = sampler.cholesky(F)
    mu = np.linspace(-3.0, 3.0, 15)
    idx = [14, 0, 3, 4, 8, 9, 10, 11, 12]
    z = workloads.standard_normals(W, D, 22)
    x = torch.empty((W, 15), dtype=torch.float64, device="cuda")
    lq = torch.empty(W, dtype=torch.float64, device="cuda")
    api.lisa_gauss_draw(_t(mu), _t(L), idx, _t(z), W, x, lq)
    xo, lqo = sampler.gauss_draw(mu, L, idx, z)
    assert np.max(np.abs(x.cpu().numpy() - xo)) <= 1e-13 * np.max(np.abs(xo))
    assert np.max(np.abs(lq.cpu().numpy() - lqo)) <= 1e-13 * np.max(np.abs(lqo))
    lq2 = torch.empty(W, dtype=torch.float64, device="cuda")
    api.lisa_gauss_logq(_t(mu), _t(L), idx, _t(xo), W, lq2)
    assert np.max(np.abs(lq2.cpu().numpy() - sampler.gauss_logq(mu, L, idx, xo))) <= 1e-12 * np.max(np.abs(lqo))


def test_gauss_walk_matches_oracle():
    D, W = 6, 500
    F = _spd(D, 23)
    L = sampler.cholesky(F)
    idx = [1, 3, 5, 7, 9, 14]
    rng = np.random.default_rng(24)
    x = rng.normal(size=(W, 15))
    z = rng.normal(size=(W, D))
    xp = torch.empty((W, 15), dtype=torch.float64, device="cuda")
    api.lisa_gauss_walk(_t(x), _t(L), idx, _t(z), W, 0.7, xp)
    want = sampler.gauss_walk(x, L, idx, z, 0.7)
    assert np.max(np.abs(xp.cpu().numpy() - want)) <= 1e-13 * np.max(np.abs(want))


def test_mh_accept_decisions_match_oracle_exactly():
    W = 4096
    rng = np.random.default_rng(31)
    x = rng.normal(size=(W, 15))
    xp = rng.normal(size=(W, 15))
    xp[::17, 4] = 5.0                                   # some proposals leave the box
    logl, loglp = rng.normal(size=W) * 3 - 10, rng.normal(size=W) * 3 - 10
    loglp[::29] = -math.inf
    logl[::31] = -math.inf
    logq, logqp = rng.normal(size=W), rng.normal(size=W)
    u = rng.uniform(1e-12, 1.0, W)
    lo, hi = np.full(15, -4.0), np.full(15, 4.0)
    xd, ld, qd = _t(x), _t(logl), _t(logq)
    acc = torch.empty(W, dtype=torch.int32, device="cuda")
    api.lisa_mh_accept(W, _t(xp), _t(loglp), _t(logqp), _t(u), lo, hi, xd, ld, qd, acc)
    xo, lo_, qo, acco = sampler.mh_accept(x, logl, logq, xp, loglp, logqp, u, lo, hi)
    assert np.array_equal(acc.cpu().numpy(), acco)
    assert np.array_equal(xd.cpu().numpy(), xo)
    assert np.array_equal(ld.cpu().numpy(), lo_) and np.array_equal(qd.cpu().numpy(), qo)
    assert 0.05 < acco.mean() < 0.95


def test_fisher_of_gpu_likelihood_matches_oracle_fisher():
    """Stencil -> GPU FP64 logL -> assemble, against the oracle's logL at the
    same points (one day, t_c and distance)."""
    cfg = workloads.config("c1_fp64_1d")
    s = oracle_setup(cfg)
    theta = workloads.c1_point()
    d = pipeline.aet(theta, s)
    idx, eps = [14, 8], np.array([0.05, 1e-3 * theta[8]])
    P = api.lisa_fisher_npoints(2)
    lk = api.Likelihood(precision=0, max_walkers=P, **gpu_kwargs(cfg))
    lk.set_data(_t(d))
    pts = torch.empty((P, 15), dtype=torch.float64, device="cuda")
    api.lisa_fisher_points(_t(theta), idx, eps, pts)
    logl = lk.loglike(pts)
    F = torch.empty((2, 2), dtype=torch.float64, device="cuda")
    api.lisa_fisher_assemble(logl, eps, F)
    Fo = sampler.fisher_assemble(np.array([pipeline.loglike(p, s, d) for p in pts.cpu().numpy()]),
                                 eps, 2)
    scale = np.sqrt(np.outer(np.diag(Fo), np.diag(Fo)))
    assert np.all(np.abs(F.cpu().numpy() - Fo) <= 1e-5 * scale)
    lk.close()


def test_tempered_accept_and_swaps_match_oracle_exactly():
    T, W = 4, 1000
    rng = np.random.default_rng(41)
    betas = np.array([1.0, 0.6, 0.3, 0.1])
    beta_w = np.repeat(betas, W)
    n = T * W
    x, xp = rng.normal(size=(n, 15)), rng.normal(size=(n, 15))
    logl, loglp = rng.normal(size=n) * 5 - 20, rng.normal(size=n) * 5 - 20
    logq, logqp = rng.normal(size=n), rng.normal(size=n)
    u = rng.uniform(1e-12, 1.0, n)
    lo, hi = np.full(15, -9.0), np.full(15, 9.0)
    xd, ld, qd = _t(x), _t(logl), _t(logq)
    acc = torch.empty(n, dtype=torch.int32, device="cuda")
    api.lisa_mh_accept(n, _t(xp), _t(loglp), _t(logqp), _t(u), lo, hi, xd, ld, qd, acc,
                       beta=_t(beta_w))
    xo, lo_, qo, acco = sampler.mh_accept(x, logl, logq, xp, loglp, logqp, u, lo, hi, beta_w)
    assert np.array_equal(acc.cpu().numpy(), acco) and np.array_equal(xd.cpu().numpy(), xo)
    us = rng.uniform(1e-12, 1.0, (T - 1) * W)
    sw = torch.empty((T - 1) * W, dtype=torch.int32, device="cuda")
    api.lisa_pt_swap(T, W, betas, _t(us), xd, ld, qd, sw)
    xs, ls, qs, swo = sampler.pt_swap(xo.reshape(T, W, 15), lo_.reshape(T, W), qo.reshape(T, W),
                                      betas, us.reshape(T - 1, W))
    assert np.array_equal(sw.cpu().numpy().reshape(T - 1, W), swo)
    assert np.array_equal(xd.cpu().numpy(), xs.reshape(n, 15))
    assert np.array_equal(ld.cpu().numpy(), ls.ravel()) and np.array_equal(qd.cpu().numpy(), qs.ravel())
    assert 0 < swo.mean() < 1
