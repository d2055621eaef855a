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
import math

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

    # checkpoint / resume: the likelihood holds no chain state, so a chain is
    # its walkers' positions, logL and log q plus the device generator's state
    def state(self):
        """The chain's state as host arrays: positions, logL, log q, the last
        acceptance flags, the walkers' inverse temperatures, the prior box and
        the device generator's state.  Restoring it and repeating the same
        steps gives the same chain bit for bit (every kernel of a step is
        deterministic and the random numbers come from the restored generator)."""
        self.torch.cuda.synchronize()
        return {"x": self.x.cpu().numpy(), "logl": self.logl.cpu().numpy(),
                "logq": self.logq.cpu().numpy(), "acc": self.acc.cpu().numpy(),
                "beta": self._betas_host(), "lo": self.lo.copy(), "hi": self.hi.copy(),
                "rng": self.gen.get_state().numpy()}

    def restore(self, st):
        """Load a state() of a chain with the same walker count, temperatures
        and prior box; raises ValueError otherwise."""
        torch = self.torch
        x = np.asarray(st["x"], dtype=np.float64)
        if x.shape != (self.W, 15):
            raise ValueError(f"checkpoint holds {x.shape[0]} walkers, this chain {self.W}")
        if not np.array_equal(np.asarray(st["beta"], dtype=np.float64), self._betas_host()):
            raise ValueError("checkpoint was taken at other temperatures")
        if not (np.array_equal(st["lo"], self.lo) and np.array_equal(st["hi"], self.hi)):
            raise ValueError("checkpoint was taken with another prior box")
        f64 = dict(dtype=torch.float64, device="cuda")
        self.x.copy_(torch.as_tensor(x, **f64))
        self.logl.copy_(torch.as_tensor(np.asarray(st["logl"], dtype=np.float64), **f64))
        self.logq.copy_(torch.as_tensor(np.asarray(st["logq"], dtype=np.float64), **f64))
        self.acc.copy_(torch.as_tensor(np.asarray(st["acc"], dtype=np.int32), device="cuda"))
        self.gen.set_state(torch.as_tensor(np.ascontiguousarray(st["rng"], dtype=np.uint8)))

    def save(self, path):
        """state() to an .npz file."""
        np.savez(path, **self.state())

    def load(self, path):
        with np.load(path) as f:
            self.restore({k: f[k] for k in f.files})

    def _betas_host(self):
        return np.ones(self.W) if self.beta is None else self.beta.cpu().numpy()

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

    def _slices(self):
        W = self.Wt
        return [slice(k * W, (k + 1) * W) for k in range(self.T)]

    def set_flow_logq(self, flows):
        """log q of every walker's state under its own temperature's flow (the
        state moves between temperatures at each exchange, so this is redone
        before every flow step)."""
        for sl, f in zip(self._slices(), flows):
            api.flow_logprob(f, self.x[sl], self.Wt, self.logq[sl])

    def step_flows(self, flows, D):
        """Independence proposals from a flow per temperature (flows[k] trained
        on temperature k's chain), the tempered MH decision on the exact
        likelihood, then replica exchange."""
        torch = self.torch
        self.set_flow_logq(flows)
        z = torch.randn((self.W, D), generator=self.gen, dtype=torch.float64, device="cuda")
        for sl, f in zip(self._slices(), flows):
            api.flow_propose(f, z[sl], self.Wt, self.xp[sl], self.logqp[sl])
        acc = self._accept(self.lik.loglike(self.xp)).clone()
        self.swap()
        return acc

    def set_gauss_logq(self, mus, Ls, idx):
        for sl, mu, L in zip(self._slices(), mus, Ls):
            api.lisa_gauss_logq(mu, L, idx, self.x[sl], self.Wt, self.logq[sl])

    def step_gauss_tempered(self, mus, Ls, idx):
        """Independence proposals N(mu_k, (L_k L_k^T)^-1) per temperature
        (the Fisher-Gaussian widened to the tempered posterior), the tempered
        MH decision, then replica exchange."""
        torch = self.torch
        self.set_gauss_logq(mus, Ls, idx)
        z = torch.randn((self.W, len(idx)), generator=self.gen, dtype=torch.float64,
                        device="cuda")
        for sl, mu, L in zip(self._slices(), mus, Ls):
            api.lisa_gauss_draw(mu, L, idx, z[sl], self.Wt, self.xp[sl], self.logqp[sl])
        acc = self._accept(self.lik.loglike(self.xp)).clone()
        self.swap()
        return acc

    def state(self):
        st = super().state()
        st["swapped"] = self.swapped.cpu().numpy()
        return st

    def restore(self, st):
        super().restore(st)
        if "swapped" in st:
            self.swapped.copy_(self.torch.as_tensor(np.asarray(st["swapped"], dtype=np.int32),
                                                    device="cuda"))

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


# parameters an aligned-spin source depends on (the tilts and spin azimuths
# of the precessing parameterisation do not enter)
ALIGNED_IDX = [0, 1, 2, 5, 8, 9, 10, 11, 12, 13, 14]
# finite-difference steps: relative for masses and distance, absolute otherwise
EPS_REL = {0: 1e-5, 1: 1e-5, 8: 1e-4}
EPS_ABS = {14: 0.05}


def fd_steps(theta):
    return np.array([EPS_REL[k] * theta[k] if k in EPS_REL else EPS_ABS.get(k, 1e-3)
                     for k in range(15)])


def fisher_diag(lik64, theta0, idx, eps):
    """The diagonal F_aa alone: the three-point stencil of each parameter
    (lisa_fisher_points with one index), all evaluated as one batch."""
    import torch
    D = len(idx)
    th = torch.as_tensor(np.asarray(theta0, dtype=np.float64), device="cuda")
    pts = torch.empty((3 * D, 15), dtype=torch.float64, device="cuda")
    for q, a in enumerate(idx):
        api.lisa_fisher_points(th, [a], [float(eps[q])], pts[3 * q:3 * q + 3])
    logl = lik64.loglike(pts)
    out = np.empty(D)
    f = torch.empty((1, 1), dtype=torch.float64, device="cuda")
    for q in range(D):
        api.lisa_fisher_assemble(logl[3 * q:3 * q + 3].contiguous(), [float(eps[q])], f)
        out[q] = float(f.item())
    return out


def fisher_scaled(lik64, theta0, idx, eps0, frac=0.3, passes=4):
    """The Fisher matrix with steps matched to the data.  Each step becomes
    frac / sqrt(F_aa), a fraction of the parameter's conditional width where
    logL is quadratic (kept within [1e-6, 10] x eps0), with F_aa from
    three-point stencils repeated until the steps settle; then the full
    stencil.  At high SNR the conditional widths of the masses are far below
    any fixed relative step, and second differences over such steps are not a
    Hessian."""
    idx = list(idx)
    e0 = np.asarray(eps0, dtype=np.float64)[idx]
    eps = e0.copy()
    for _ in range(passes):
        d = fisher_diag(lik64, theta0, idx, eps)
        new = np.where(d > 0, frac / np.sqrt(np.where(d > 0, d, 1.0)), eps)
        new = np.clip(new, 1e-6 * e0, 10.0 * e0)
        done = np.all(np.abs(np.log(new / eps)) < math.log(1.5))
        eps = new
        if done:
            break
    return fisher(lik64, theta0, idx, eps)


def box_around(theta, tc_halfwidth=600.0):
    """A broad uniform box around theta (masses and distance within a factor
    of two, spins within [-0.99, 0.99], angles over their full ranges, the
    merger time +- tc_halfwidth): the prior widths that regularise the Fisher
    matrix along directions the data leave unconstrained."""
    th = np.asarray(theta, dtype=np.float64)
    lo = np.array([0.5 * th[0], 0.5 * th[1], -0.99, 0.0, -np.pi, -0.99, 0.0, -np.pi,
                   0.5 * th[8], 0.0, 0.0, -0.5 * np.pi, 0.0, 0.0, th[14] - tc_halfwidth])
    hi = np.array([2.0 * th[0], 2.0 * th[1], 0.99, np.pi, np.pi, 0.99, np.pi, np.pi,
                   2.0 * th[8], np.pi, 2.0 * np.pi, 0.5 * np.pi, 2.0 * np.pi, np.pi,
                   th[14] + tc_halfwidth])
    return lo, hi


def fisher_ball(lik64, theta0, idx, count, seed, lo=None, hi=None):
    """`count` draws theta ~ N(theta0, (F + diag(12/w^2))^-1) in the parameters
    idx (the others stay at theta0): the posterior bulk around an injection at
    theta0, from the FP64 likelihood's Fisher matrix.  -> device [count][15]."""
    import torch
    if lo is None:
        lo, hi = box_around(theta0)
    F = fisher_scaled(lik64, theta0, idx, fd_steps(np.asarray(theta0, dtype=np.float64)))
    L = gauss_factor(F, idx, lo, hi)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    D = len(idx)
    z = torch.randn((count, D), generator=gen, dtype=torch.float64, device="cuda")
    mu = torch.as_tensor(np.asarray(theta0, dtype=np.float64), device="cuda")
    x = torch.empty((count, 15), dtype=torch.float64, device="cuda")
    q = torch.empty(count, dtype=torch.float64, device="cuda")
    api.lisa_gauss_draw(mu, L, idx, z, count, x, q)
    # keep the draws inside the box (spins must stay below 1 in magnitude)
    x = torch.maximum(torch.minimum(x, torch.as_tensor(hi, device="cuda")),
                      torch.as_tensor(lo, device="cuda"))
    return x.contiguous()


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
