"""Contexts on the caller's orbit table (orbit_kind 2, lisa_td_create_orbits):
the spacecraft positions of a mission orbit file (Sec. II.B, orbits; the
unequal-arm runs of Sec. III.C), resampled by the library and, independently,
by the oracle."""
import dataclasses

import numpy as np
import pytest

from oracle import orbits, pipeline
from oracle import consts as K
from paper_2501_08261_gb300 import api, workloads

from helpers import gpu_kwargs, oracle_setup

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2501_08261_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


T0, DT_TAB = -2 * 3600.0, 3600.0


def _table(cfg, seed=3):
    rows = int((cfg["n"] * cfg["dt"] - T0) // DT_TAB) + 10
    return workloads.orbit_table_positions(T0, DT_TAB, rows, seed)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["c2_hm_1d", "c3_prec_1d"])
def test_orbit_table_context_matches_oracle(name, precision):
    cfg = workloads.config(name, orbit=2)
    pos = _table(cfg)
    s = dataclasses.replace(oracle_setup(workloads.config(name)),
                            orbit=orbits.OrbitTable(T0, DT_TAB, pos))
    th = workloads.prior_draws(3, cfg["n"], cfg["dt"], 41, precessing=bool(cfg["precessing"]),
                               logm=(5.5, 7.0))
    lk = api.Likelihood(precision=precision, max_walkers=3, orbit_table=(T0, DT_TAB, pos),
                        **gpu_kwargs(cfg))
    aet = lk.tdi(lk.project(_t(th))).cpu().numpy()
    tol = 1e-10 if precision == 0 else 1e-4
    d = pipeline.aet(th[0], s)
    for w in range(3):
        want = pipeline.aet(th[w], s) if w else d
        # relative to the largest channel (TDI 2's T is suppressed far below A
        # and E, and rounding of the retarded times scales with the signal, not
        # with T).  The mixed path's FP32 h carries a white rounding floor of
        # ~1e-7 |h|; the link tests bound each y by 1e-4 max(|y|, 1e-2 |h|), and
        # A, E, T add at most 32 / sqrt 2, 64 / sqrt 6 and 48 / sqrt 3 (< 28)
        # such y errors (16 terms per TDI-2 channel), so the floor of their bar
        # is 28 x 1e-6 |h|: it matters for heavy sources, whose A, E, T at a few
        # mHz TDI suppresses to < 1e-2 |h| while the rounding noise sits at high
        # frequencies where TDI passes it with gain ~16
        bar = tol * np.max(np.abs(want))
        if precision == 1:
            hp, hc = pipeline.polarizations(th[w], s)
            bar = max(bar, 28.0 * 1e-6 * max(np.max(np.abs(hp)), np.max(np.abs(hc))))
        for c in range(3):
            assert np.max(np.abs(aet[c, :, w] - want[c])) <= bar, (w, c)
    # logL against the injection of walker 0 at SNR 500
    far = th[0].copy()
    far[8] = 1e30
    rho = np.sqrt(-2.0 * pipeline.loglike(far, s, d))
    d = d * (500.0 / rho)
    th[0, 8] *= rho / 500.0
    lk.set_data(_t(d))
    got = lk.loglike(_t(th)).cpu().numpy()
    for w in range(3):
        o = pipeline.loglike(th[w], s, d)
        bar = max(1e-6, 1e-11 * abs(o)) if precision == 0 else max(0.05, 1e-4 * abs(o))
        assert abs(got[w] - o) <= bar, (w, got[w], o)
    lk.close()


def test_keplerian_positions_through_the_table_equal_the_keplerian_model():
    """The built-in Keplerian orbits tabulated hourly and passed as a table
    give the A, E, T and logL of orbit_kind 1 (FP64), up to the table's
    resampling error."""
    cfg1 = workloads.config("c2_hm_1d")
    rows = int((cfg1["n"] * cfg1["dt"] - T0) // DT_TAB) + 10
    tt = T0 + DT_TAB * np.arange(rows)
    pos = np.stack([orbits.kepler_position(k, tt) for k in (1, 2, 3)], axis=1) * K.C_SI
    th = workloads.prior_draws(4, cfg1["n"], cfg1["dt"], 42, logm=(5.5, 7.0))
    lk1 = api.Likelihood(precision=0, max_walkers=4, **gpu_kwargs(cfg1))
    lk2 = api.Likelihood(precision=0, max_walkers=4, orbit_table=(T0, DT_TAB, pos),
                         **gpu_kwargs(dict(cfg1, orbit=2)))
    a1 = lk1.tdi(lk1.project(_t(th))).cpu().numpy()
    a2 = lk2.tdi(lk2.project(_t(th))).cpu().numpy()
    for w in range(4):
        scale = np.max(np.abs(a1[:, :, w]))
        for c in range(3):
            assert np.max(np.abs(a2[c, :, w] - a1[c, :, w])) <= 1e-9 * scale, (w, c)
    d = _t(a1[:, :, 0])
    lk1.set_data(d)
    lk2.set_data(d)
    l1, l2 = lk1.loglike(_t(th)).cpu().numpy(), lk2.loglike(_t(th)).cpu().numpy()
    assert np.all(np.abs(l1 - l2) <= np.maximum(1e-6, 1e-8 * np.abs(l1))), (l1, l2)
    lk1.close()
    lk2.close()
