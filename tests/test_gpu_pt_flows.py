"""Parallel tempering with a flow per temperature (the ptemcee-like sampler of
Sec. II.C with its temperatures): each temperature's flow, trained on that
temperature's Fisher random-walk chain, is accepted more often than the
Fisher-Gaussian widened to the same temperature, at every temperature, and
more often than the Fisher random walk at every beta < 1, with every proposal
judged by the exact likelihood."""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu]
torch = pytest.importorskip("torch")


def test_flow_per_temperature_beats_the_tempered_fisher_gaussian():
    from paper_2501_08261_gb300 import build, proposals
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    r = proposals.compare_tempered()
    acc_f = np.array(r["flow"]["acceptance"])
    acc_g = np.array(r["fisher_gauss"]["acceptance"])
    acc_w = np.array(r["fisher_random_walk"]["acceptance"])
    assert np.all(acc_f > acc_g), r
    # and above the Fisher random walk that trained it, at every beta < 1
    assert np.all(acc_f[1:] > acc_w[1:]), r
    assert r["flow"]["ess_cold_per_s"] > r["fisher_gauss"]["ess_cold_per_s"], r
