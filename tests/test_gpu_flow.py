"""Parity of the tensor-core flow kernels (include/lisa_flow.h) with the
oracle flow (oracle/flow.py): against the oracle with the same bfloat16
operand rounding (tight: fp32 accumulation order, tanh/exp rounding and rare
bf16 rounding-boundary flips remain) and against the plain FP64 oracle (the
error bfloat16 operands cost)."""
import numpy as np
import pytest

from oracle import flow as oflow
from paper_2501_08261_gb300 import api

pytestmark = [pytest.mark.gpu]
torch = pytest.importorskip("torch")

D, L, H = 15, 6, 128
IDX = [0, 1, 2, 5, 8, 9, 10, 11, 12, 13, 14, 3, 4, 6, 7]


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2501_08261_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def make(seed, max_batch=1024):
    rng = np.random.default_rng(seed)
    perms = np.stack([rng.permutation(D) for _ in range(L)])
    of = oflow.Flow(D, L, H, perms)
    theta = np.concatenate([
        np.concatenate([(rng.normal(size=np.prod(s)) * (0.1 if n.startswith("b") else
                                                         (0.12 if n == "W3" else 0.3 / np.sqrt(s[-1]))))
                        for n, s in of.shapes(l)]) for l in range(L)])
    theta = theta.astype(np.float32).astype(np.float64)      # the GPU keeps fp32 masters
    f = api.flow_create(D, L, H, max_batch, IDX, perms)
    assert api.flow_nparams(f) == of.n_params()
    api.flow_set_params(f, _t(theta, torch.float32))
    mu = rng.normal(size=15)
    scale = rng.uniform(0.5, 2.0, D)
    api.flow_set_frame(f, _t(mu), _t(scale))
    return f, of, theta, mu, scale, rng


def test_params_round_trip():
    f, of, theta, *_ = make(1)
    back = torch.empty(of.n_params(), dtype=torch.float32, device="cuda")
    api.flow_get_params(f, back)
    assert np.array_equal(back.cpu().numpy().astype(np.float64), theta)
    api.flow_destroy(f)


@pytest.mark.parametrize("W", [1, 128, 300])
def test_logprob_matches_oracle(W):
    f, of, theta, mu, scale, rng = make(2)
    x = np.repeat(mu[None], W, axis=0)
    x[:, IDX] += rng.normal(size=(W, D)) * scale * 1.3
    lq = torch.empty(W, dtype=torch.float64, device="cuda")
    api.flow_logprob(f, _t(x), W, lq)
    got = lq.cpu().numpy()
    u, lj = oflow.to_frame(x, IDX, mu, scale)
    em = of.logq_u(theta, u, bf16=True) + lj
    ex = of.logq_u(theta, u, bf16=False) + lj
    assert np.all(np.isfinite(got))
    # same bf16 operands: fp32 accumulation / tanh / exp rounding, plus rare
    # rounding-boundary flips of a bf16 operand (one 2^-8 step) -> tight in
    # bulk, 2e-3 at worst
    err = np.abs(got - em)
    assert np.percentile(err, 90) <= 1e-4 and np.max(err) <= 2e-3, (np.percentile(err, 90), err.max())
    # against FP64: no further from it than bf16 operands themselves put the oracle
    assert np.max(np.abs(got - ex)) <= 1.5 * np.max(np.abs(em - ex)) + 2e-3
    api.flow_destroy(f)


def test_propose_matches_oracle_inverse_and_round_trips():
    W = 300
    f, of, theta, mu, scale, rng = make(3)
    z = rng.normal(size=(W, D))
    x = torch.empty((W, 15), dtype=torch.float64, device="cuda")
    lq = torch.empty(W, dtype=torch.float64, device="cuda")
    api.flow_propose(f, _t(z), W, x, lq)
    xg = x.cpu().numpy()
    u, ld = of.inverse(theta, z, bf16=True)
    xo = oflow.from_frame(u, IDX, mu, scale)
    lqo = (-0.5 * np.sum(z * z, axis=1) - 0.5 * D * np.log(2 * np.pi) + ld
           - np.sum(np.log(scale)))
    ex = np.abs(xg - xo)[:, IDX] / scale
    assert np.percentile(ex, 90) <= 1e-5 and np.max(ex) <= 5e-3, (np.percentile(ex, 90), ex.max())
    el = np.abs(lq.cpu().numpy() - lqo)
    assert np.percentile(el, 90) <= 1e-4 and np.max(el) <= 5e-3, (np.percentile(el, 90), el.max())
    # density of the proposals equals the log q the proposal reported
    lq2 = torch.empty(W, dtype=torch.float64, device="cuda")
    api.flow_logprob(f, x, W, lq2)
    assert np.max(np.abs(lq2.cpu().numpy() - lq.cpu().numpy())) <= 1e-3
    api.flow_destroy(f)


def test_zero_parameters_are_the_identity_map():
    rng = np.random.default_rng(4)
    perms = np.stack([rng.permutation(D) for _ in range(L)])
    f = api.flow_create(D, L, H, 256, IDX, perms)
    mu = rng.normal(size=15)
    scale = rng.uniform(0.5, 2.0, D)
    api.flow_set_frame(f, _t(mu), _t(scale))
    z = rng.normal(size=(200, D))
    x = torch.empty((200, 15), dtype=torch.float64, device="cuda")
    lq = torch.empty(200, dtype=torch.float64, device="cuda")
    api.flow_propose(f, _t(z), 200, x, lq)
    want = oflow.from_frame(z.astype(np.float32).astype(np.float64), IDX, mu, scale)
    assert np.max(np.abs(x.cpu().numpy() - want)) <= 1e-12 * np.max(np.abs(want))
    api.flow_destroy(f)


def _split(of, g):
    """packed vector -> list of (layer, name, block)"""
    out, k = [], 0
    for l in range(L):
        for name, shp in of.shapes(l):
            m = int(np.prod(shp))
            out.append((l, name, g[k:k + m]))
            k += m
    return out


@pytest.mark.parametrize("B", [128, 300])
def test_gradient_matches_oracle_backprop(B):
    f, of, theta, mu, scale, rng = make(5)
    x = np.repeat(mu[None], B, axis=0)
    x[:, IDX] += rng.normal(size=(B, D)) * scale
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    grad = torch.empty(of.n_params(), dtype=torch.float32, device="cuda")
    api.flow_grad(f, _t(x), B, loss, grad)
    g = grad.cpu().numpy().astype(np.float64)
    u, lj = oflow.to_frame(x, IDX, mu, scale)
    g_em = of.grad(theta, u, bf16=True)
    g64 = of.grad(theta, u, bf16=False)
    assert np.all(np.isfinite(g))
    assert loss.item() == pytest.approx(of.loss(theta, u, bf16=True) - lj, rel=1e-4)
    assert np.linalg.norm(g - g_em) <= 5e-3 * np.linalg.norm(g_em), np.linalg.norm(g - g_em) / np.linalg.norm(g_em)
    for (l, name, a), (_, _, b) in zip(_split(of, g), _split(of, g_em)):
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-6, (l, name)
    assert np.linalg.norm(g - g64) <= 1.5 * np.linalg.norm(g_em - g64) + 5e-3 * np.linalg.norm(g64)
    api.flow_destroy(f)


def test_adam_step_matches_oracle():
    f, of, theta, mu, scale, rng = make(6)
    n = of.n_params()
    g1 = rng.normal(size=n).astype(np.float32).astype(np.float64)
    g2 = rng.normal(size=n).astype(np.float32).astype(np.float64)
    for g in (g1, g2):
        api.flow_adam(f, _t(g, torch.float32), 1e-3)
    th, m, v = theta.copy(), np.zeros(n), np.zeros(n)
    th, m, v = oflow.adam_step(th, m, v, g1, 1, 1e-3)
    th, m, v = oflow.adam_step(th, m, v, g2, 2, 1e-3)
    back = torch.empty(n, dtype=torch.float32, device="cuda")
    api.flow_get_params(f, back)
    assert np.max(np.abs(back.cpu().numpy() - th)) <= 1e-6 * max(1.0, np.max(np.abs(th)))
    api.flow_destroy(f)


def test_training_fits_a_curved_distribution():
    """Samples of a banana-shaped density in 15 dimensions: after training the
    flow's mean log-density on held-out samples beats the best Gaussian's."""
    rng = np.random.default_rng(7)
    S = 16384
    def draw(n):
        y = rng.normal(size=(n, D))
        y[:, 1] = y[:, 1] * 0.3 + 0.8 * (y[:, 0] ** 2 - 1.0)      # curved pair
        y[:, 3] = y[:, 3] * 0.2 + 0.9 * np.sin(1.5 * y[:, 2])      # another
        x = np.zeros((n, 15))
        x[:, IDX] = y
        return x
    xs, xt = draw(S), draw(4096)
    perms = np.stack([rng.permutation(D) for _ in range(L)])
    f = api.flow_create(D, L, H, 8192, IDX, perms)
    init = np.concatenate([
        np.concatenate([(rng.normal(size=np.prod(s)) * (0.0 if n in ("W3", "b3") else
                                                        (0.0 if n.startswith("b") else 1.0 / np.sqrt(s[-1]))))
                        for n, s in oflow.Flow(D, L, H, perms).shapes(l)]) for l in range(L)])
    api.flow_set_params(f, _t(init, torch.float32))
    api.flow_set_frame(f, _t(np.zeros(15)), _t(np.ones(D)))
    losses = torch.empty(30, dtype=torch.float32, device="cuda")
    api.flow_train(f, _t(xs), S, 30, 1024, 2e-3, losses)
    lv = losses.cpu().numpy()
    lq = torch.empty(4096, dtype=torch.float64, device="cuda")
    api.flow_logprob(f, _t(xt), 4096, lq)
    flow_ll = lq.cpu().numpy().mean()
    yt = xt[:, IDX]
    mean, cov = xs[:, IDX].mean(axis=0), np.cov(xs[:, IDX].T)
    from scipy.stats import multivariate_normal
    gauss_ll = multivariate_normal(mean, cov).logpdf(yt).mean()
    assert np.all(np.isfinite(lv)) and lv[-1] < lv[0] - 1.0, lv
    assert flow_ll > gauss_ll + 0.5, (flow_ll, gauss_ll)
    api.flow_destroy(f)
