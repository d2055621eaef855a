"""lisa_td_noise against the oracle's noise synthesis (same normals), and the
likelihood of noisy data: at the true parameters logL = -1/2 (n|n), which is
-1/2 of the sum of the band's squared normals."""
import numpy as np
import pytest

from oracle import noise, pipeline
from paper_2501_08261_gb300 import api, workloads

from helpers import gpu_kwargs, norm_rel, oracle_setup

pytestmark = [pytest.mark.gpu]
torch = pytest.importorskip("torch")


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("gen", [15, 20])
def test_noise_matches_oracle_and_gives_chi2_loglike(gen):
    from paper_2501_08261_gb300 import build
    build.build()
    cfg = workloads.config("c2_hm_1d", tdi_gen=gen)
    n, dt = cfg["n"], cfg["dt"]
    nb = n // 2 + 1
    z = np.random.default_rng(gen).normal(size=(3, 2, nb))
    lk = api.Likelihood(precision=0, max_walkers=2, **gpu_kwargs(cfg))
    out = torch.empty((3, n), dtype=torch.float64, device="cuda")
    api.lisa_td_noise(lk.ctx, _t(z), out)
    got = out.cpu().numpy()
    want = noise.noise_aet(z, n, dt, cfg["f_lo"], cfg["f_hi"], gen)
    for c in range(3):
        assert norm_rel(got[c], want[c]) < 1e-10, c
    # noisy data: signal of walker 0 plus the noise; logL at the truth = -1/2 (n|n)
    th = workloads.prior_draws(2, n, dt, 90, logm=(5.5, 6.5))
    s = oracle_setup(cfg)
    sig = pipeline.aet(th[0], s)
    lk.set_data(_t(sig + got))
    ll = lk.loglike(_t(th)).cpu().numpy()
    mask = (np.arange(nb) / (n * dt) >= cfg["f_lo"]) & (np.arange(nb) / (n * dt) <= cfg["f_hi"])
    chi2 = float(np.sum(z[:, :, mask] ** 2))
    assert ll[0] == pytest.approx(-0.5 * chi2, rel=1e-9)
    o = pipeline.loglike(th[1], s, sig + want)
    assert abs(ll[1] - o) <= max(1e-6, 1e-11 * abs(o))
    lk.close()
