"""lisa_td_autotune: the tuned launch shapes are valid and leave the
likelihood unchanged (up to the rounding of the projection's FP32 tile
anchors), for the batch path and for ragged batches."""
import numpy as np
import pytest

from paper_2501_08261_gb300 import api, workloads

from helpers import gpu_kwargs

pytestmark = [pytest.mark.gpu]
torch = pytest.importorskip("torch")
DAY = 17280


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_keeps_the_likelihood(precision):
    from paper_2501_08261_gb300 import build
    build.build()
    cfg = workloads.config("c2_hm_1d", n=4 * DAY)
    W = 40
    th = workloads.prior_draws(W, cfg["n"], 5.0, 3, logm=(5.5, 6.5))
    windows = np.array(([4, 2, 1, 3] * 10)[:W]) * DAY
    th[:, 14] = cfg["n"] * 5.0 - 0.1 * windows * 5.0
    plain = api.Likelihood(precision=precision, max_walkers=W + 32, **gpu_kwargs(cfg))
    tuned = api.Likelihood(precision=precision, max_walkers=W + 32, **gpu_kwargs(cfg))
    d = plain.tdi(plain.project(_t(th[:1])))[:, :, 0].to(torch.float64).contiguous()
    # the mixed path's |dlogL| <= 0.05 holds at SNR 2000 (louder injections
    # move the truth walker's logL by rounding alone, ~ SNR^2): scale to it
    plain.set_data(d)
    far0 = th[:1].copy()
    far0[0, 8] = 1e30
    rho = float(np.sqrt(-2.0 * plain.loglike(_t(far0)).cpu().numpy()[0]))
    d = (d * (2000.0 / rho)).contiguous()
    th[0, 8] *= rho / 2000.0
    plain.set_data(d)
    tuned.set_data(d)
    choice = api.lisa_td_autotune(tuned.ctx, _t(th), W, windows)
    assert choice[0] in (64, 128, 256) and choice[2] in (1, 2, 4, 8, 16) and choice[3] in (1, 2, 4, 8, 16)
    assert choice[1] == (0 if precision == 0 else choice[1]) and (precision == 0 or choice[1] in (4, 8))
    assert choice[4] in (256, 512) and choice[5] in (256, 512)
    a, b = plain.loglike(_t(th)).cpu().numpy(), tuned.loglike(_t(th)).cpu().numpy()
    ra = plain.loglike_ragged(_t(th), windows).cpu().numpy()
    rb = tuned.loglike_ragged(_t(th), windows).cpu().numpy()
    far = th.copy()
    far[:, 8] = 1e30
    dd = np.abs(plain.loglike(_t(far)).cpu().numpy())
    for x, y in ((a, b), (ra, rb)):
        if precision == 0:
            bar = np.maximum(1e-6, 1e-10 * np.sqrt(4.0 * np.abs(x) * dd) + 1e-10 * np.abs(x))
        else:
            # a different FFT block shape regroups FP32 rounding: the mixed
            # path's own bar (the injection walker's logL is rounding noise)
            bar = np.maximum(0.05, 1e-4 * np.abs(x))
        assert np.all(np.abs(x - y) <= bar), np.max(np.abs(x - y) / bar)
    plain.close()
    tuned.close()
