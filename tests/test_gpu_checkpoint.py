"""Checkpoint and resume of the sampler (the likelihood holds no chain state):
a tempered chain saved to .npz and loaded into a new chain continues bit for
bit as the uninterrupted one, a checkpoint of another shape or ladder is
refused, and a flow restored from its saved parameters and frame scores and
proposes exactly as the original."""
import math

import numpy as np
import pytest

from paper_2501_08261_gb300 import api, mcmc, proposals, workloads

pytestmark = [pytest.mark.gpu]
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2501_08261_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def test_tempered_chain_resumes_bit_for_bit(tmp_path):
    cfg = workloads.config("c3_prec_1d")
    kw = {k: cfg[k] for k in ("dt", "n", "t0", "f_lo", "f_hi", "tdi_gen", "channel_mask",
                              "lagrange_order", "orbit", "mode_mask", "precessing")}
    truth = workloads.table1_precessing(cfg["n"], cfg["dt"], tc_frac=0.75)
    idx = list(range(15))
    lo, hi = workloads.table1_prior_box(truth[14])
    T, W = 2, 64
    lik64 = api.Likelihood(precision=0, max_walkers=api.lisa_fisher_npoints(15), **kw)
    lik = api.Likelihood(precision=1, max_walkers=T * W, **kw)
    d = lik64.tdi(lik64.project(_t(truth[None])))[:, :, 0].contiguous()
    lik64.set_data(d)
    lik.set_data(d)
    L = mcmc.gauss_factor(mcmc.fisher(lik64, truth, idx, proposals.fd_steps(truth)), idx, lo, hi)
    betas = mcmc.geometric_ladder(T, 1e-2)
    step = 2.38 / math.sqrt(15)
    pt = mcmc.PT(lik, lo, hi, W, betas, seed=5)
    x0 = torch.empty((T * W, 15), dtype=torch.float64, device="cuda")
    q0 = torch.empty(T * W, dtype=torch.float64, device="cuda")
    z = torch.randn((T * W, 15), generator=torch.Generator(device="cuda").manual_seed(3),
                    dtype=torch.float64, device="cuda")
    api.lisa_gauss_draw(_t(truth), L, idx, z, T * W, x0, q0)
    pt.start(torch.minimum(torch.maximum(x0, _t(lo)), _t(hi)).contiguous())
    for _ in range(6):
        pt.step_walk(L, idx, step)
    path = str(tmp_path / "chain.npz")
    pt.save(path)
    for _ in range(6):
        pt.step_walk(L, idx, step)
    want = [a.cpu().numpy() for a in (pt.x, pt.logl, pt.logq, pt.swapped)]
    # another seed: the generator's state comes from the checkpoint
    pt2 = mcmc.PT(lik, lo, hi, W, betas, seed=99)
    pt2.load(path)
    for _ in range(6):
        pt2.step_walk(L, idx, step)
    got = [a.cpu().numpy() for a in (pt2.x, pt2.logl, pt2.logq, pt2.swapped)]
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    assert np.all(np.isfinite(want[1]))
    with pytest.raises(ValueError, match="temperatures"):
        mcmc.PT(lik, lo, hi, W, mcmc.geometric_ladder(T, 1e-3), seed=1).load(path)
    with pytest.raises(ValueError, match="walkers"):
        mcmc.MH(lik, lo, hi, W, seed=1).load(path)
    lik.close()
    lik64.close()


def test_restored_flow_scores_and_proposes_identically(tmp_path):
    rng = np.random.default_rng(11)
    D, layers, H, W = 15, 4, 128, 256
    idx = list(range(D))
    perms = np.stack([rng.permutation(D) for _ in range(layers)])
    p0 = proposals.flow_init(perms, D, layers, H, 7)
    p0 = (p0 + 0.02 * rng.standard_normal(p0.size)).astype(np.float32)
    mu, scale = rng.normal(size=15), rng.uniform(0.5, 2.0, D)
    fl = api.flow_create(D, layers, H, W, idx, perms)
    api.flow_set_params(fl, torch.as_tensor(p0, device="cuda"))
    api.flow_set_frame(fl, _t(mu), _t(scale))
    path = str(tmp_path / "flow.npz")
    np.savez(path, **proposals.flow_state(fl, D, layers, H, idx, perms, mu, scale))
    with np.load(path) as f:
        fl2 = proposals.flow_from_state({k: f[k] for k in f.files}, W)
    x = _t(mu + rng.normal(size=(W, 15)))
    z = _t(rng.normal(size=(W, D)))
    out = []
    for f in (fl, fl2):
        q = torch.full((W,), float("nan"), dtype=torch.float64, device="cuda")
        xp = torch.empty((W, 15), dtype=torch.float64, device="cuda")
        qp = torch.empty(W, dtype=torch.float64, device="cuda")
        api.flow_logprob(f, x, W, q)
        api.flow_propose(f, z, W, xp, qp)
        torch.cuda.synchronize()
        out.append([a.cpu().numpy() for a in (q, xp, qp)])
    for a, b in zip(*out):
        assert np.all(np.isfinite(a)) and np.array_equal(a, b)
    api.flow_destroy(fl)
    api.flow_destroy(fl2)
