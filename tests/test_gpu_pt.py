"""Parallel tempering on the exact likelihood (one-day precessing Table I
injection): replica exchange happens, the chains stay finite and inside the
prior, and the colder the temperature the higher the logL the chain holds."""
import math

import numpy as np
import pytest

from paper_2501_08261_gb300 import api, mcmc, proposals, workloads

pytestmark = [pytest.mark.gpu]
torch = pytest.importorskip("torch")


def test_parallel_tempering_orders_the_temperatures():
    from paper_2501_08261_gb300 import build
    build.build()
    cfg = workloads.config("c3_prec_1d")
    kw = {k: cfg[k] for k in ("dt", "n", "t0", "f_lo", "f_hi", "tdi_gen", "channel_mask",
                              "lagrange_order", "orbit", "mode_mask", "precessing")}
    truth = workloads.table1_precessing(cfg["n"], cfg["dt"], tc_frac=0.75)
    idx = list(range(15))
    lo, hi = workloads.table1_prior_box(truth[14])
    T, W = 4, 128
    T_ = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    lik64 = api.Likelihood(precision=0, max_walkers=api.lisa_fisher_npoints(15), **kw)
    lik = api.Likelihood(precision=1, max_walkers=T * W, **kw)
    d = lik64.tdi(lik64.project(T_(truth[None])))[:, :, 0].contiguous()
    lik64.set_data(d)
    lik.set_data(d)
    F = mcmc.fisher(lik64, truth, idx, proposals.fd_steps(truth))
    L = mcmc.gauss_factor(F, idx, lo, hi)
    betas = mcmc.geometric_ladder(T, 1e-3)
    pt = mcmc.PT(lik, lo, hi, W, betas, seed=5)
    x0 = torch.empty((T * W, 15), dtype=torch.float64, device="cuda")
    q0 = torch.empty(T * W, dtype=torch.float64, device="cuda")
    z = torch.randn((T * W, 15), dtype=torch.float64, device="cuda")
    api.lisa_gauss_draw(T_(truth), L, idx, z, T * W, x0, q0)
    x0 = torch.minimum(torch.maximum(x0, T_(lo)), T_(hi)).contiguous()   # start inside the prior
    pt.start(x0)
    nsw = 0
    for it in range(150):
        pt.step_walk(L, idx, 2.38 / math.sqrt(15))
        nsw += int(pt.swapped[:(T - 1) * W].sum().item())
    logl = pt.logl.cpu().numpy().reshape(T, W)
    x = pt.x.cpu().numpy()
    assert np.all(np.isfinite(logl)) and nsw > 0
    assert np.all(x >= lo - 1e-9) and np.all(x <= hi + 1e-9)
    med = np.median(logl, axis=1)
    assert np.all(np.diff(med) < 0), med
    lik.close()
    lik64.close()
