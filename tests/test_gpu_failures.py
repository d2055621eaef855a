"""Failure paths that need no GPU fault (host-side injection and bounded
device waits that are made to give up):

* a workspace allocation of lisa_td_create fails (LISA_TD_FAIL_ALLOC): the
  call returns LISA_TD_ENOMEM, frees what it had allocated, and a following
  create and likelihood call work;
* the flow kernels' waits on their tensor-core work give up at once
  (flow_set_wait_limit(f, 0)): the kernel drains its product in flight and
  frees its tensor memory, the next call reports LISA_TD_ETIMEOUT, and with
  the default limit restored the flow computes log q as before."""
import numpy as np
import pytest

from paper_2501_08261_gb300 import api, workloads

from helpers import gpu_kwargs

pytestmark = [pytest.mark.gpu]
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2501_08261_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def test_allocation_failure_is_reported_and_cleaned_up(monkeypatch):
    cfg = workloads.config("c1_fp64_1d")
    free0 = torch.cuda.mem_get_info()[0]
    for k in (0, 5, 12):
        monkeypatch.setenv("LISA_TD_FAIL_ALLOC", str(k))
        with pytest.raises(api.LisaTdError, match="ENOMEM"):
            api.Likelihood(precision=1, max_walkers=64, **gpu_kwargs(cfg))
    monkeypatch.delenv("LISA_TD_FAIL_ALLOC")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)    # nothing leaked
    th = workloads.prior_draws(4, cfg["n"], cfg["dt"], 5, logm=(5.5, 7.0))
    lk = api.Likelihood(precision=1, max_walkers=4, **gpu_kwargs(cfg))
    lk.set_data(torch.zeros((3, cfg["n"]), dtype=torch.float64, device="cuda"))
    got = lk.loglike(torch.as_tensor(th, device="cuda")).cpu().numpy()
    assert np.all(np.isfinite(got)) and np.all(got < 0)
    lk.close()


def test_flow_wait_that_gives_up_reports_etimeout_and_recovers():
    from oracle import flow as oflow
    rng = np.random.default_rng(9)
    D, L, W = 15, 3, 300
    perms = np.stack([rng.permutation(D) for _ in range(L)])
    of = oflow.Flow(D, L, 128, perms)
    theta = (rng.normal(size=of.n_params()) * 0.05).astype(np.float32).astype(np.float64)
    f = api.flow_create(D, L, 128, 512, list(range(D)), perms)
    api.flow_set_params(f, torch.as_tensor(theta, dtype=torch.float32, device="cuda"))
    x = torch.as_tensor(rng.normal(size=(W, 15)), device="cuda")
    lq = torch.full((W,), float("nan"), dtype=torch.float64, device="cuda")
    api.flow_set_wait_limit(f, 0)
    api.flow_logprob(f, x, W, lq)               # every CTA gives up at its first wait
    torch.cuda.synchronize()
    api.flow_set_wait_limit(f, -1)
    with pytest.raises(api.LisaTdError, match="ETIMEOUT"):
        api.flow_logprob(f, x, W, lq)
    api.flow_logprob(f, x, W, lq)               # the mark was cleared: a normal call
    torch.cuda.synchronize()
    want = of.logq_u(theta, x.cpu().numpy(), bf16=True)
    assert np.max(np.abs(lq.cpu().numpy() - want)) <= 2e-3
    api.flow_destroy(f)
