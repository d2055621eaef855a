"""Batched Metropolis-Hastings driver over the C ABI (host orchestration only).

Every arithmetic step runs in the library's kernels: the likelihood
(lisa_td_loglike_batch), the proposals (lisa_gauss_walk, lisa_gauss_draw,
flow_propose) and the decision (lisa_mh_accept).  This module draws the
random numbers (torch generators on the device; the kernels take them as
inputs), keeps the chain state in device tensors and records the chain.

Sec. II.C of arXiv:2501.08261: the Fisher matrix is built from finite
differences of the likelihood at the injection and the sampler starts from
N(theta_inj, F^-1).  Here that Gaussian is also the baseline independence
proposal, a random walk with the Fisher covariance generates the chain the
flow learns from, and the trained flow is the learned independence proposal.
``ess`` is the effective sample size from the integrated autocorrelation
time with Sokal's automatic window (analysis of recorded chains, host side).
"""
import numpy as np

from . import api


class MH:
    """W walkers of an MH chain on the likelihood `lik` inside the box [lo, hi]."""

    def __init__(self, lik, lo, hi, W, seed=0, beta=None):
        import torch
        self.torch = torch
        self.lik, self.W = lik, W
        # inverse temperature of each walker (tempered targets pi^beta), or None
        self.beta = None if beta is None else torch.as_tensor(beta, dtype=torch.float64,
                                                              device="cuda").contiguous()
        self.lo, self.hi = np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)
        self.gen = torch.Generator(device="cuda")
        self.gen.manual_seed(seed)
        f64 = dict(dtype=torch.float64, device="cuda")
        self.x = torch.empty((W, 15), **f64)
        self.logl = torch.empty(W, **f64)
        self.logq = torch.zeros(W, **f64)
        self.xp = torch.empty((W, 15), **f64)
        self.logqp = torch.zeros(W, **f64)
        self.acc = torch.zeros(W, dtype=torch.int32, device="cuda")

    def start(self, x0, logq0=None):
        self.x.copy_(x0)
        self.logl.copy_(self.lik.loglike(self.x))
        if logq0 is None:
            self.logq.zero_()
        else:
            self.logq.copy_(logq0)

    def _accept(self, loglp):
        u = self.torch.rand(self.W, generator=self.gen, dtype=self.torch.float64, device="cuda")
        u = 1.0 - u                                        # (0, 1]
        api.lisa_mh_accept(self.W, self.xp, loglp, self.logqp, u, self.lo, self.hi, self.x,
                           self.logl, self.logq, self.acc, beta=self.beta)
        return self.acc

    def step_walk(self, L, idx, step):
        """Random walk with covariance step^2 F^-1 (symmetric: log q = 0)."""
        z = self.torch.randn((self.W, len(idx)), generator=self.gen, dtype=self.torch.float64,
                             device="cuda")
        api.lisa_gauss_walk(self.x, L, idx, z, self.W, step, self.xp)
        self.logqp.zero_()
        return self._accept(self.lik.loglike(self.xp))

    def step_gauss(self, mu, L, idx):
        """Independence proposal N(mu, (L L^T)^-1)."""
        z = self.torch.randn((self.W, len(idx)), generator=self.gen, dtype=self.torch.float64,
                             device="cuda")
        api.lisa_gauss_draw(mu, L, idx, z, self.W, self.xp, self.logqp)
        return self._accept(self.lik.loglike(self.xp))

    def step_flow(self, flow, D):
        """Independence proposal from a trained flow (lisa_flow.h)."""
        z = self.torch.randn((self.W, D), generator=self.gen, dtype=self.torch.float64,
                             device="cuda")
        api.flow_propose(flow, z, self.W, self.xp, self.logqp)
        return self._accept(self.lik.loglike(self.xp))

    def set_gauss_logq(self, mu, L, idx):
        api.lisa_gauss_logq(mu, L, idx, self.x, self.W, self.logq)

    def set_flow_logq(self, flow):
        api.flow_logprob(flow, self.x, self.W, self.logq)

    def run(self, step_fn, steps, record=None):
        """`steps` MH steps; returns (chain [steps][W][15] host array or None,
        mean acceptance, GPU milliseconds measured with CUDA events)."""
        torch = self.torch
        chain = np.empty((steps, self.W, 15)) if record else None
        dev = torch.empty((steps, self.W, 15), dtype=torch.float64, device="cuda") if record else None
        acc = torch.zeros(self.W, dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for it in range(steps):
            a = step_fn()
            acc += a
            if record:
                dev[it].copy_(self.x)
        e1.record()
        torch.cuda.synchronize()
        if record:
            chain[:] = dev.cpu().numpy()
        return chain, float(acc.mean().item()) / steps, e0.elapsed_time(e1)


class PT(MH):
    """Parallel tempering (the sampler of Sec. II.C is ptemcee): T temperatures
    x W walkers in one batch, temperature-major, betas[0] = 1; each step is an
    MH step of every walker at its temperature followed by replica exchange
    between adjacent temperatures (lisa_pt_swap)."""

    def __init__(self, lik, lo, hi, W, betas, seed=0):
        self.T = len(betas)
        self.betas = np.asarray(betas, dtype=np.float64)
        super().__init__(lik, lo, hi, self.T * W, seed, beta=np.repeat(self.betas, W))
        self.Wt = W
        self.swapped = self.torch.zeros(self.T * W, dtype=self.torch.int32, device="cuda")

    def step_walk(self, L, idx, step):
        """Fisher random walk at every temperature, the step widened by
        1/sqrt(beta) (the tempered posterior's width), then replica exchange."""
        torch = self.torch
        z = torch.randn((self.W, len(idx)), generator=self.gen, dtype=torch.float64,
                        device="cuda")
        W = self.Wt
        for k in range(self.T):
            sl = slice(k * W, (k + 1) * W)
            api.lisa_gauss_walk(self.x[sl], L, idx, z[sl], W, step / np.sqrt(self.betas[k]),
                                self.xp[sl])
        self.logqp.zero_()
        acc = self._accept(self.lik.loglike(self.xp)).clone()
        self.swap()
        return acc

    def swap(self):
        torch = self.torch
        u = 1.0 - torch.rand((self.T - 1) * self.Wt, generator=self.gen, dtype=torch.float64,
                             device="cuda")
        api.lisa_pt_swap(self.T, self.Wt, self.betas, u, self.x, self.logl, self.logq,
                         self.swapped)
        return self.swapped[:(self.T - 1) * self.Wt]


def geometric_ladder(T, beta_min):
    """betas[k] = beta_min^(k / (T - 1)), k = 0 .. T-1 (ptemcee's default shape)."""
    return beta_min ** (np.arange(T) / max(T - 1, 1))


def fisher(lik64, theta0, idx, eps):
    """F [D][D] on the device from the stencil of lisa_fisher_points evaluated
    with the FP64 likelihood `lik64` (max_walkers >= lisa_fisher_npoints(D))."""
    import torch
    D = len(idx)
    P = api.lisa_fisher_npoints(D)
    th = torch.as_tensor(np.asarray(theta0, dtype=np.float64), device="cuda")
    pts = torch.empty((P, 15), dtype=torch.float64, device="cuda")
    api.lisa_fisher_points(th, idx, eps, pts)
    logl = lik64.loglike(pts)
    F = torch.empty((D, D), dtype=torch.float64, device="cuda")
    api.lisa_fisher_assemble(logl, eps, F)
    return F


def gauss_factor(F, idx, lo, hi):
    """Cholesky factor of F + diag(12 / w^2) (w = prior widths of idx)."""
    import torch
    D = len(idx)
    w = (np.asarray(hi) - np.asarray(lo))[idx]
    L = torch.empty((D, D), dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    api.lisa_cholesky(F, D, L, info, diag=12.0 / w ** 2)
    if int(info.item()) != 0:
        raise RuntimeError(f"Fisher matrix not positive definite (column {int(info.item())})")
    return L


def integrated_time(y, c=5.0):
    """Integrated autocorrelation time of y [N][W] (one parameter, W walkers):
    the walkers' normalised autocorrelation functions averaged, summed up to
    Sokal's automatic window M >= c tau(M)."""
    y = np.asarray(y, dtype=np.float64)
    N = y.shape[0]
    yc = y - y.mean(axis=0, keepdims=True)
    n2 = 1 << (2 * N - 1).bit_length()
    f = np.fft.rfft(yc, n=n2, axis=0)
    acf = np.fft.irfft(f * np.conj(f), n=n2, axis=0)[:N]
    var = acf[0]
    ok = var > 0
    if not np.any(ok):
        return float(N)                                 # a chain that never moved
    rho = (acf[:, ok] / var[ok]).mean(axis=1)
    taus = 2.0 * np.cumsum(rho) - 1.0
    m = np.arange(N)
    win = np.nonzero(m >= c * taus)[0]
    return float(taus[win[0]] if len(win) else taus[-1])


def ess(chain, idx):
    """Effective samples of a recorded chain [N][W][15]: N W / max_i tau_i."""
    N, W = chain.shape[0], chain.shape[1]
    tau = max(integrated_time(chain[:, :, k]) for k in idx)
    return N * W / max(tau, 1.0), tau
