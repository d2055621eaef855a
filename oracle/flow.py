"""Affine-coupling normalising flow used as the sampler's learned proposal.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's sampler starts from, and is judged against, the Fisher-Gaussian
proposal (Sec. II.C).  The learned proposal replaces that Gaussian by a
RealNVP-style flow (Dinh, Sohl-Dickstein & Bengio 2017): an invertible map
u -> z built from L coupling layers.  Layer l splits its input by a fixed
permutation perm_l into a conditioning part a (the first d_a entries) and a
transformed part b (the rest); an MLP of the a-part gives (s_raw, t) and
    y_a = u_a,   y_b = u_b * exp(s) + t,   s = tanh(s_raw),
with the MLP  h1 = tanh(W1 u_a + b1),  h2 = tanh(W2 h1 + b2),
(s_raw, t) = W3 h2 + b3.  Parameters u are the sampled physical parameters
in a fixed frame, u = (x[idx] - mu[idx]) / scale.  The density is
    log q(x) = sum_i [-z_i^2/2 - log(2 pi)/2] + sum_l sum_b s_l - sum_i log scale_i,
and a proposal is drawn by z ~ N(0, I) and the inverse layers
u_b = (y_b - t) exp(-s).  Training minimises the mean of -log q over
samples by back-propagation and Adam (Kingma & Ba 2015; beta1 0.9,
beta2 0.999, eps 1e-8, bias-corrected).

``bf16=True`` rounds every matrix-product operand (u_a, W1, W2, W3, h1, h2 in
the forward pass; the back-propagated matrix and the transposed activations
in the backward pass) to bfloat16 with round-to-nearest-even, as the
tensor-core kernels do, the products then summed in FP64; with ``bf16=False``
everything is FP64.  Parameter packing per layer (FP32 master copy on the
GPU): W1 [H][d_a], b1 [H], W2 [H][H], b2 [H], W3 [2 d_b][H], b3 [2 d_b],
rows of W3 / b3 ordered s first, then t.
"""
import math

import numpy as np


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if np.any(nan):
        out = np.where(nan, np.nan, out)
    return out


class Flow:
    def __init__(self, dim, layers, hidden, perms):
        self.D, self.L, self.H = dim, layers, hidden
        self.perm = np.asarray(perms, dtype=np.int64).reshape(layers, dim)
        self.da = [dim // 2 + (dim % 2) if l % 2 == 0 else dim // 2 for l in range(layers)]

    def db(self, l):
        return self.D - self.da[l]

    def shapes(self, l):
        da, db, H = self.da[l], self.db(l), self.H
        return [("W1", (H, da)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
                ("W3", (2 * db, H)), ("b3", (2 * db,))]

    def n_params(self):
        return sum(int(np.prod(s)) for l in range(self.L) for _, s in self.shapes(l))

    def unpack(self, theta):
        theta = np.asarray(theta, dtype=np.float64)
        out, k = [], 0
        for l in range(self.L):
            p = {}
            for name, s in self.shapes(l):
                m = int(np.prod(s))
                p[name] = theta[k:k + m].reshape(s)
                k += m
            out.append(p)
        return out

    # -- one coupling layer ------------------------------------------------
    def _mlp(self, p, ua, bf16):
        q = bf16_round if bf16 else (lambda v: v)
        pre1 = q(ua) @ q(p["W1"]).T + p["b1"]
        h1 = np.tanh(pre1)
        pre2 = q(h1) @ q(p["W2"]).T + p["b2"]
        h2 = np.tanh(pre2)
        out = q(h2) @ q(p["W3"]).T + p["b3"]
        return pre1, h1, pre2, h2, out

    def forward(self, theta, u, bf16=False, keep=False):
        """u [N][D] -> z [N][D], sum of s [N]; keep: per-layer caches."""
        params = self.unpack(theta)
        z = np.array(u, dtype=np.float64)
        logdet = np.zeros(len(z))
        caches = []
        for l in range(self.L):
            p, perm, da = params[l], self.perm[l], self.da[l]
            ia, ib = perm[:da], perm[da:]
            ua, ub = z[:, ia], z[:, ib]
            pre1, h1, pre2, h2, out = self._mlp(p, ua, bf16)
            db = len(ib)
            s = np.tanh(out[:, :db])
            t = out[:, db:]
            yb = ub * np.exp(s) + t
            if keep:
                caches.append(dict(ua=ua, ub=ub, h1=h1, h2=h2, s=s))
            z = z.copy()
            z[:, ib] = yb
            logdet += s.sum(axis=1)
        return (z, logdet, caches) if keep else (z, logdet)

    def inverse(self, theta, z, bf16=False):
        """z [N][D] -> u [N][D] and the sum of s [N] (log q uses +sum s)."""
        params = self.unpack(theta)
        u = np.array(z, dtype=np.float64)
        logdet = np.zeros(len(u))
        for l in reversed(range(self.L)):
            p, perm, da = params[l], self.perm[l], self.da[l]
            ia, ib = perm[:da], perm[da:]
            out = self._mlp(p, u[:, ia], bf16)[4]
            db = len(ib)
            s = np.tanh(out[:, :db])
            t = out[:, db:]
            u = u.copy()
            u[:, ib] = (u[:, ib] - t) * np.exp(-s)
            logdet += s.sum(axis=1)
        return u, logdet

    def logq_u(self, theta, u, bf16=False):
        z, logdet = self.forward(theta, u, bf16)
        return -0.5 * np.sum(z * z, axis=1) - 0.5 * self.D * math.log(2 * math.pi) + logdet

    def loss(self, theta, u, bf16=False):
        return -float(np.mean(self.logq_u(theta, u, bf16)))

    def grad(self, theta, u, bf16=False):
        """d loss / d theta by back-propagation (packed like theta)."""
        q = bf16_round if bf16 else (lambda v: v)
        params = self.unpack(theta)
        N = len(u)
        z, logdet, caches = self.forward(theta, u, bf16, keep=True)
        dz = z / N                                    # d(mean |z|^2/2)
        grads = [None] * self.L
        for l in reversed(range(self.L)):
            p, perm, da, c = params[l], self.perm[l], self.da[l], caches[l]
            ia, ib = perm[:da], perm[da:]
            dyb, dya = dz[:, ib], dz[:, ia]
            es = np.exp(c["s"])
            ds = dyb * c["ub"] * es - 1.0 / N          # -mean(sum s) term
            dsr = ds * (1.0 - c["s"] ** 2)
            dout = np.concatenate([dsr, dyb], axis=1)  # [N][2 db]
            g = {}
            g["W3"] = q(dout).T @ q(c["h2"])
            g["b3"] = dout.sum(axis=0)
            dh2 = q(dout) @ q(p["W3"])
            dpre2 = dh2 * (1.0 - c["h2"] ** 2)
            g["W2"] = q(dpre2).T @ q(c["h1"])
            g["b2"] = dpre2.sum(axis=0)
            dh1 = q(dpre2) @ q(p["W2"])
            dpre1 = dh1 * (1.0 - c["h1"] ** 2)
            g["W1"] = q(dpre1).T @ q(c["ua"])
            g["b1"] = dpre1.sum(axis=0)
            dua = q(dpre1) @ q(p["W1"])
            dprev = dz.copy()
            dprev[:, ia] = dya + dua
            dprev[:, ib] = dyb * es
            dz = dprev
            grads[l] = g
        return np.concatenate([grads[l][name].ravel() for l in range(self.L)
                               for name, _ in self.shapes(l)])


def adam_step(theta, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step count t >= 1); returns new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def to_frame(x, idx, mu, scale):
    """u = (x[idx] - mu[idx]) / scale, and the frame's log-Jacobian -sum log scale."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    return (x[:, idx] - np.asarray(mu)[idx]) / scale, -float(np.sum(np.log(scale)))


def from_frame(u, idx, mu, scale):
    u = np.atleast_2d(u)
    x = np.repeat(np.asarray(mu, dtype=np.float64)[None, :], len(u), axis=0)
    x[:, idx] = np.asarray(mu)[idx] + u * scale
    return x
