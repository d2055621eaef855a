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

# finite-difference steps: relative for masses and distance, absolute otherwise
EPS_REL = {0: 1e-5, 1: 1e-5, 8: 1e-4}
EPS_ABS = {14: 0.05}


def fd_steps(theta):
    return np.array([EPS_REL[k] * theta[k] if k in EPS_REL else EPS_ABS.get(k, 1e-3)
                     for k in range(15)])


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
    F = mcmc.fisher(lik64, truth, idx, fd_steps(truth))
    L = mcmc.gauss_factor(F, idx, lo, hi)
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
    return {
        "workload": f"{cfg_name}: 1 d @ 5 s, precessing, 5 modes, Keplerian, TDI 2; Table I "
                    f"injection (SNR {snr:.0f}), {W} walkers, {D} parameters, uniform Table I priors",
        "fisher_random_walk": {"acceptance": acc_rw, "steps": rw_steps, "tau": tau_rw,
                               "ess": ess_rw, "gpu_ms": ms_rw},
        "fisher_gauss": {"acceptance": acc_g, "steps": steps, "tau": tau_g, "ess": ess_g,
                         "gpu_ms": ms_g, "ess_per_s": ess_g / (ms_g * 1e-3)},
        "flow": {"acceptance": acc_f, "steps": steps, "tau": tau_f, "ess": ess_f,
                 "gpu_ms": ms_f, "ess_per_s": ess_f / (ms_f * 1e-3),
                 "train_ms": train_ms, "train_samples": len(samples), "epochs": epochs,
                 "loss_first_last": [float(lv[0]), float(lv[-1])]},
    }
