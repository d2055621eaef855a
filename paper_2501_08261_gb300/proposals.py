"""The learned-proposal experiment: Fisher-Gaussian vs flow independence
proposals on the exact likelihood (host orchestration over the C ABI).

Sequence (Sec. II.C's Fisher initialization, then the learned proposal):
Fisher matrix at the injection from the FP64 likelihood, a random-walk chain
with the Fisher covariance (the chain the flow learns from), the flow trained
on that chain, then two independence chains of the same length -- proposals
from N(theta_inj, F^-1) and from the flow -- each accepted or rejected by the
exact (mixed-precision) likelihood.  Reports acceptance rates, effective
samples and effective samples per second of GPU time.
"""
import math

import numpy as np

from . import api, mcmc, workloads

fd_steps = mcmc.fd_steps


def flow_init(perms, D, L, H, seed):
    """Initial flow parameters: W1, W2 ~ N(0, 1/fan_in), zero biases and zero
    output layer (the flow starts as the identity map)."""
    rng = np.random.default_rng(seed)
    out = []
    for l in range(L):
        da = (D + 1) // 2 if l % 2 == 0 else D // 2
        db = D - da
        out += [rng.normal(size=H * da) / math.sqrt(da), np.zeros(H),
                rng.normal(size=H * H) / math.sqrt(H), np.zeros(H),
                np.zeros(2 * db * H), np.zeros(2 * db)]
    return np.concatenate(out).astype(np.float32)


def flow_state(fl, D, layers, hidden, idx, perms, mu, scale):
    """A trained flow as host arrays: its shape, coupling masks, frame (mu [15],
    scale [D]: the library keeps them write-only, so the caller passes the ones
    it set) and parameters from flow_get_params.  The optimiser's moments are
    not kept: a restored flow proposes and scores; training starts afresh."""
    import torch
    params = torch.empty(api.flow_nparams(fl), dtype=torch.float32, device="cuda")
    api.flow_get_params(fl, params)
    torch.cuda.synchronize()
    return {"D": np.int64(D), "layers": np.int64(layers), "hidden": np.int64(hidden),
            "idx": np.asarray(idx, dtype=np.int32), "perms": np.asarray(perms, dtype=np.int32),
            "mu": np.asarray(mu, dtype=np.float64), "scale": np.asarray(scale, dtype=np.float64),
            "params": params.cpu().numpy()}


def flow_from_state(st, max_batch):
    """A new flow context from flow_state() (or the arrays of its .npz file)."""
    import torch
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    fl = api.flow_create(int(st["D"]), int(st["layers"]), int(st["hidden"]), max_batch,
                         [int(i) for i in st["idx"]], np.asarray(st["perms"]))
    api.flow_set_params(fl, torch.as_tensor(np.ascontiguousarray(st["params"], dtype=np.float32),
                                            device="cuda"))
    api.flow_set_frame(fl, T(st["mu"]), T(st["scale"]))
    return fl


def compare(cfg_name="c3_prec_1d", W=512, rw_steps=600, burn=100, steps=600, epochs=40,
            batch=4096, lr=1e-3, layers=6, seed=1):
    import torch
    cfg = workloads.config(cfg_name)
    kw = {k: cfg[k] for k in ("dt", "n", "t0", "f_lo", "f_hi", "tdi_gen", "channel_mask",
                              "lagrange_order", "orbit", "mode_mask", "precessing")}
    truth = workloads.table1_precessing(cfg["n"], cfg["dt"], tc_frac=0.75)
    idx = list(range(15))
    D = len(idx)
    lo, hi = workloads.table1_prior_box(truth[14])
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    lik64 = api.Likelihood(precision=0, max_walkers=api.lisa_fisher_npoints(D), **kw)
    lik = api.Likelihood(precision=1, max_walkers=W, **kw)
    d = lik64.tdi(lik64.project(T(truth[None])))[:, :, 0].contiguous()
    lik64.set_data(d)
    lik.set_data(d)
    far = truth.copy()
    far[8] = 1e30
    snr = math.sqrt(-2.0 * lik64.loglike(T(far[None])).item())
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    # the fixed relative steps first (at one day they give the proposal the
    # sampler mixes best with); where the signal is long enough that those steps
    # leave the quadratic region and the matrix is indefinite, steps scaled to
    # each parameter's conditional width
    try:
        F = mcmc.fisher(lik64, truth, idx, fd_steps(truth))
        L = mcmc.gauss_factor(F, idx, lo, hi)
    except RuntimeError:
        F = mcmc.fisher_scaled(lik64, truth, idx, fd_steps(truth))
        L = mcmc.gauss_factor(F, idx, lo, hi)
    f1.record()
    torch.cuda.synchronize()
    fisher_ms = f0.elapsed_time(f1)
    mu = T(truth)
    ch = mcmc.MH(lik, lo, hi, W, seed=seed)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed + 100)
    x0 = torch.empty((W, 15), dtype=torch.float64, device="cuda")
    q0 = torch.empty(W, dtype=torch.float64, device="cuda")
    api.lisa_gauss_draw(mu, L, idx, torch.randn((W, D), generator=gen, dtype=torch.float64,
                                                 device="cuda"), W, x0, q0)
    ch.start(x0)
    rw, acc_rw, ms_rw = ch.run(lambda: ch.step_walk(L, idx, 2.38 / math.sqrt(D)), rw_steps,
                               record=True)
    ess_rw, tau_rw = mcmc.ess(rw[burn:], idx)
    # flow trained on the random-walk chain after burn-in
    samples = rw[burn:].reshape(-1, 15)
    rng = np.random.default_rng(seed + 200)
    perms = np.stack([rng.permutation(D) for _ in range(layers)])
    fl = api.flow_create(D, layers, 128, max(W, batch), idx, perms)
    api.flow_set_params(fl, torch.as_tensor(flow_init(perms, D, layers, 128, seed + 300),
                                            device="cuda"))
    api.flow_set_frame(fl, T(samples.mean(axis=0)), T(samples[:, idx].std(axis=0)))
    losses = torch.empty(epochs, dtype=torch.float32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    api.flow_train(fl, T(samples), len(samples), epochs, batch, lr, losses)
    e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    start = ch.x.clone()
    ch.start(start)
    ch.set_gauss_logq(mu, L, idx)
    gc, acc_g, ms_g = ch.run(lambda: ch.step_gauss(mu, L, idx), steps, record=True)
    ess_g, tau_g = mcmc.ess(gc, idx)
    ch.start(start)
    ch.set_flow_logq(fl)
    fc, acc_f, ms_f = ch.run(lambda: ch.step_flow(fl, D), steps, record=True)
    ess_f, tau_f = mcmc.ess(fc, idx)
    api.flow_destroy(fl)
    lik.close()
    lik64.close()
    lv = losses.cpu().numpy()
    days = cfg["n"] * cfg["dt"] / 86400.0
    # amortised over the training: the flow's chain charged with its training
    # time (the Fisher-Gaussian needs none); and over the whole protocol: every
    # GPU millisecond, the Fisher matrix and the random-walk chain included --
    # both protocols run that chain first, so its own effective samples count
    # for both (and, on short signals, dominate both)
    t_g = fisher_ms + ms_rw + ms_g
    t_f = fisher_ms + ms_rw + train_ms + ms_f
    return {
        "workload": f"{cfg_name}: {days:g} d @ {cfg['dt']:g} s, precessing, 5 modes, Keplerian, "
                    f"TDI 2; Table I injection (SNR {snr:.0f}), {W} walkers, {D} parameters, "
                    f"uniform Table I priors; flow trained on {len(samples)} chain samples",
        "fisher_ms": fisher_ms,
        "amortised": {"fisher_gauss_ess_per_s": ess_g / (ms_g * 1e-3),
                      "flow_ess_per_s": ess_f / ((ms_f + train_ms) * 1e-3),
                      "note": "ESS of the proposal's chain / (chain [+ training] GPU time)"},
        "protocol": {"fisher_gauss_ess_per_s": (ess_rw + ess_g) / (t_g * 1e-3),
                     "flow_ess_per_s": (ess_rw + ess_f) / (t_f * 1e-3),
                     "note": "(ESS of the random-walk chain + ESS of the proposal's chain) / "
                             "(Fisher + random walk [+ training] + chain GPU time)"},
        "fisher_random_walk": {"acceptance": acc_rw, "steps": rw_steps, "tau": tau_rw,
                               "ess": ess_rw, "gpu_ms": ms_rw},
        "fisher_gauss": {"acceptance": acc_g, "steps": steps, "tau": tau_g, "ess": ess_g,
                         "gpu_ms": ms_g, "ess_per_s": ess_g / (ms_g * 1e-3)},
        "flow": {"acceptance": acc_f, "steps": steps, "tau": tau_f, "ess": ess_f,
                 "gpu_ms": ms_f, "ess_per_s": ess_f / (ms_f * 1e-3),
                 "train_ms": train_ms, "train_samples": len(samples), "epochs": epochs,
                 "loss_first_last": [float(lv[0]), float(lv[-1])]},
    }


def _train_flow(samples, idx, layers, epochs, batch, lr, seed, max_batch):
    """A flow on `samples` [S][15] (host), trained on the tensor cores: -> (flow,
    training GPU ms)."""
    import torch
    D = len(idx)
    rng = np.random.default_rng(seed)
    perms = np.stack([rng.permutation(D) for _ in range(layers)])
    fl = api.flow_create(D, layers, 128, max(max_batch, batch), idx, perms)
    api.flow_set_params(fl, torch.as_tensor(flow_init(perms, D, layers, 128, seed + 1),
                                            device="cuda"))
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    api.flow_set_frame(fl, T(samples.mean(axis=0)), T(samples[:, idx].std(axis=0) + 1e-300))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    api.flow_train(fl, T(samples), len(samples), epochs, batch, lr, None)
    e1.record()
    torch.cuda.synchronize()
    return fl, e0.elapsed_time(e1)


def _pt_run(pt, step, steps, record=False):
    """`steps` tempered steps: -> (acceptance per temperature [T], cold-chain
    record [steps][W][15] or None, GPU ms)."""
    import torch
    T, W = pt.T, pt.Wt
    acc = torch.zeros(T * W, dtype=torch.float64, device="cuda")
    cold = torch.empty((steps, W, 15), dtype=torch.float64, device="cuda") if record else None
    allx = torch.empty((steps, T * W, 15), dtype=torch.float64, device="cuda") if record == "all" else None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for it in range(steps):
        acc += step()
        if record:
            cold[it].copy_(pt.x[:W])
        if allx is not None:
            allx[it].copy_(pt.x)
    e1.record()
    torch.cuda.synchronize()
    rate = (acc.view(T, W).mean(dim=1) / steps).cpu().numpy()
    out = allx.cpu().numpy() if allx is not None else (cold.cpu().numpy() if record else None)
    return rate, out, e0.elapsed_time(e1)


def compare_tempered(cfg_name="c3_prec_1d", T=4, W=256, beta_min=1e-3, rw_steps=600, burn=200,
                     steps=200, epochs=40, batch=4096, lr=1e-3, layers=6, seed=2):
    """Parallel tempering with a flow per temperature (the ptemcee-like
    sampler of Sec. II.C with T temperatures): a Fisher random walk at every
    temperature generates each temperature's training chain, one flow is
    trained per temperature, and the tempered independence chains of the flows
    and of the per-temperature Fisher-Gaussians N(theta_inj, F^-1 / beta) run
    from the same state, every proposal judged by the exact likelihood and
    replicas exchanged after each step.  Reports acceptance per temperature
    and the cold chain's effective samples per second."""
    import torch
    cfg = workloads.config(cfg_name)
    kw = {k: cfg[k] for k in ("dt", "n", "t0", "f_lo", "f_hi", "tdi_gen", "channel_mask",
                              "lagrange_order", "orbit", "mode_mask", "precessing")}
    truth = workloads.table1_precessing(cfg["n"], cfg["dt"], tc_frac=0.75)
    idx = list(range(15))
    D = len(idx)
    lo, hi = workloads.table1_prior_box(truth[14])
    Tt = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    lik64 = api.Likelihood(precision=0, max_walkers=api.lisa_fisher_npoints(D), **kw)
    lik = api.Likelihood(precision=1, max_walkers=T * W, **kw)
    d = lik64.tdi(lik64.project(Tt(truth[None])))[:, :, 0].contiguous()
    lik64.set_data(d)
    lik.set_data(d)
    F = mcmc.fisher(lik64, truth, idx, fd_steps(truth))
    L = mcmc.gauss_factor(F, idx, lo, hi)
    betas = mcmc.geometric_ladder(T, beta_min)
    pt = mcmc.PT(lik, lo, hi, W, betas, seed=seed)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed + 100)
    x0 = torch.empty((T * W, 15), dtype=torch.float64, device="cuda")
    q0 = torch.empty(T * W, dtype=torch.float64, device="cuda")
    api.lisa_gauss_draw(Tt(truth), L, idx, torch.randn((T * W, D), generator=gen,
                                                        dtype=torch.float64, device="cuda"),
                        T * W, x0, q0)
    x0 = torch.minimum(torch.maximum(x0, Tt(lo)), Tt(hi)).contiguous()
    pt.start(x0)
    acc_rw, rw, ms_rw = _pt_run(pt, lambda: pt.step_walk(L, idx, 2.38 / math.sqrt(D)),
                                rw_steps, record="all")
    flows, train_ms = [], 0.0
    for k in range(T):
        samples = rw[burn:, k * W:(k + 1) * W].reshape(-1, 15)
        fl, ms = _train_flow(samples, idx, layers, epochs, batch, lr, seed + 10 * k, T * W)
        flows.append(fl)
        train_ms += ms
    start = pt.x.clone()
    mus = [Tt(truth)] * T
    Ls = [(L * math.sqrt(b)).contiguous() for b in betas]
    pt.start(start)
    acc_g, gc, ms_g = _pt_run(pt, lambda: pt.step_gauss_tempered(mus, Ls, idx), steps,
                              record=True)
    ess_g, tau_g = mcmc.ess(gc, idx)
    pt.start(start)
    acc_f, fc, ms_f = _pt_run(pt, lambda: pt.step_flows(flows, D), steps, record=True)
    ess_f, tau_f = mcmc.ess(fc, idx)
    for fl in flows:
        api.flow_destroy(fl)
    lik.close()
    lik64.close()
    return {
        "workload": f"{cfg_name}: Table I precessing injection, {T} temperatures "
                    f"(geometric ladder to beta = {beta_min:g}) x {W} walkers, {D} parameters",
        "betas": [float(b) for b in betas],
        "fisher_random_walk": {"acceptance": [float(a) for a in acc_rw], "steps": rw_steps,
                               "gpu_ms": ms_rw},
        "fisher_gauss": {"acceptance": [float(a) for a in acc_g], "steps": steps, "tau": tau_g,
                         "ess_cold": ess_g, "ess_cold_per_s": ess_g / (ms_g * 1e-3)},
        "flow": {"acceptance": [float(a) for a in acc_f], "steps": steps, "tau": tau_f,
                 "ess_cold": ess_f, "ess_cold_per_s": ess_f / (ms_f * 1e-3),
                 "train_ms": train_ms,
                 "ess_cold_per_s_amortised": ess_f / ((ms_f + train_ms + ms_rw) * 1e-3)},
    }
