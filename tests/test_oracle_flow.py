"""Pins of the oracle's affine-coupling flow: bfloat16 rounding against the
library conversion and hand-checked ties, exact invertibility, the density
against a brute-force Jacobian determinant, back-propagation against finite
differences, and Adam's closed-form first step."""
import math

import numpy as np
import pytest

from oracle import flow


def _flow(D=5, L=4, H=8, seed=0):
    rng = np.random.default_rng(seed)
    perms = np.stack([rng.permutation(D) for _ in range(L)])
    f = flow.Flow(D, L, H, perms)
    theta = rng.normal(size=f.n_params()) * 0.4
    return f, theta, rng


def test_bf16_rounding_ties_and_library():
    one = 1.0
    assert flow.bf16_round(one) == 1.0
    assert flow.bf16_round(1 + 2.0 ** -8) == 1.0                    # tie -> even (down)
    assert flow.bf16_round(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6      # tie -> even (up)
    assert flow.bf16_round(1 + 2.0 ** -8 + 2.0 ** -20) == 1 + 2.0 ** -7
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(1).normal(size=10000) * 10.0 ** np.random.default_rng(2).uniform(-8, 8, 10000)
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(flow.bf16_round(x), want)


@pytest.mark.parametrize("bf16", [False, True])
def test_inverse_undoes_forward(bf16):
    f, theta, rng = _flow()
    u = rng.normal(size=(200, 5))
    z, ld = f.forward(theta, u, bf16)
    u2, ld2 = f.inverse(theta, z, bf16)
    assert np.max(np.abs(u2 - u)) < 1e-11
    assert np.max(np.abs(ld2 - ld)) < 1e-11


def test_density_matches_bruteforce_jacobian():
    f, theta, rng = _flow(D=4, L=3, H=6, seed=3)
    u = rng.normal(size=(5, 4))
    lq = f.logq_u(theta, u)
    h = 1e-6
    for n in range(len(u)):
        J = np.zeros((4, 4))
        for j in range(4):
            up, um = u[n].copy(), u[n].copy()
            up[j] += h
            um[j] -= h
            J[:, j] = (f.forward(theta, up[None])[0][0] - f.forward(theta, um[None])[0][0]) / (2 * h)
        z = f.forward(theta, u[n][None])[0][0]
        want = -0.5 * z @ z - 2.0 * math.log(2 * math.pi) + math.log(abs(np.linalg.det(J)))
        assert abs(lq[n] - want) < 1e-7


def test_backprop_matches_finite_differences():
    f, theta, rng = _flow(D=5, L=4, H=8, seed=4)
    u = rng.normal(size=(64, 5))
    g = f.grad(theta, u)
    h = 1e-6
    pick = rng.choice(len(theta), 60, replace=False)
    for k in pick:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (f.loss(tp, u) - f.loss(tm, u)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), k


def test_bf16_gradient_close_to_fp64_gradient():
    # at initialisation-sized weights (std 0.1) the bfloat16 operands move the
    # gradient by a few 1e-3 of its norm (unit roundoff 2^-9 per operand)
    f, theta, rng = _flow(D=15, L=6, H=32, seed=5)
    theta *= 0.25
    u = rng.normal(size=(256, 15))
    g64, g16 = f.grad(theta, u), f.grad(theta, u, bf16=True)
    assert np.linalg.norm(g16 - g64) <= 1e-2 * np.linalg.norm(g64)


def test_adam_first_step_is_signed_lr():
    g = np.array([3.0, -2e-3, 0.5])
    th, m, v = flow.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, 0.01)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=1e-5)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_frame_round_trip():
    rng = np.random.default_rng(6)
    mu = rng.normal(size=15)
    idx = [1, 4, 14]
    scale = np.array([2.0, 0.5, 10.0])
    u = rng.normal(size=(7, 3))
    x = flow.from_frame(u, idx, mu, scale)
    u2, lj = flow.to_frame(x, idx, mu, scale)
    assert np.allclose(u2, u, atol=1e-13) and lj == pytest.approx(-math.log(10.0))
