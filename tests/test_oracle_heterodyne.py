"""Pins of the heterodyned time-domain likelihood in ``oracle/heterodyne.py``
against what fixes it independently of its own code: the polarisations of
``waveform.plus_cross``, the one-sided spectrum an analytic signal must have,
the sampled (Lagrange) response of ``pipeline.aet``, the exactness of the
construction at the fiducial and with a node at every sample, the
fourth-order convergence of cubic interpolation, and the node rule's accuracy
and spacing.  CPU only."""

import numpy as np
import pytest

from oracle import heterodyne as H
from oracle import likelihood, pipeline, waveform
from paper_2501_08261_gb300 import workloads as wl

DAY = 86400.0


def _setup(precessing=False, n=17280, **kw):
    base = dict(dt=5.0, n=n, t0=0.0, tdi_gen=20, orbit="kepler", mode_mask=31,
                precessing=precessing)
    base.update(kw)
    return pipeline.Setup(**base)


def _theta(precessing=False, tc=None, seed=3):
    th = wl.c1_point(seed)
    th[8] = 20.0
    if precessing:
        th[2], th[3], th[4] = 0.6, 1.0, 0.5
        th[5], th[6], th[7] = 0.3, 2.0, 1.0
    if tc is not None:
        th[14] = tc
    return th


def _nearby(th, scale=1.0):
    """A point about one posterior width away (SNR ~ 10^3) in several parameters."""
    q = th.copy()
    q[14] += 0.05 * scale
    q[0] *= 1.0 + 2e-5 * scale
    q[10] += 1e-3 * scale
    q[11] += 1e-4 * scale
    return q


@pytest.mark.parametrize("precessing", [False, True])
def test_analytic_modes_sum_to_the_polarisations(precessing):
    s = _setup(precessing)
    th = _theta(precessing)
    t = np.linspace(0.0, 0.8 * DAY, 4001)
    hp, hc = waveform.plus_cross(th, t, s.t0, s.mode_mask, precessing)
    am = H.analytic_modes(th, t, s)
    assert len(am) == 5
    sp = sum(a[2] for a in am)
    sx = sum(a[3] for a in am)
    assert np.max(np.abs(sp.real - hp)) <= 1e-13 * np.max(np.abs(hp))
    assert np.max(np.abs(sx.real - hc)) <= 1e-13 * np.max(np.abs(hc))


@pytest.mark.parametrize("precessing", [False, True])
def test_analytic_modes_have_one_sided_spectra(precessing):
    """h_lm = A e^{-i Phi} with Phi rising: each analytic polarisation must put
    its power at negative frequencies (numpy's e^{-2 pi i f t} convention).  A
    wrong quadrature (a conjugate or a sign of i dropped) moves half of it to
    positive frequencies while leaving the real parts unchanged."""
    s = _setup(precessing)
    th = _theta(precessing)
    t = 0.3 * DAY + 5.0 * np.arange(8192)          # inspiral, well before merger
    win = np.sin(np.pi * np.arange(8192) / 8191.0) ** 4
    for (l, m, hp, hx) in H.analytic_modes(th, t, s):
        for sig in (hp, hx):
            F = np.fft.fft(sig * win)
            f = np.fft.fftfreq(t.size, 5.0)
            pos = np.sum(np.abs(F[f > 0]) ** 2)
            neg = np.sum(np.abs(F[f < 0]) ** 2)
            assert pos <= 1e-8 * neg, (l, m, pos / neg)


def test_mode_phase_is_the_phase_of_the_mode():
    th = _theta()
    src = waveform.source(th, False)
    t = np.linspace(0.0, 0.8 * DAY, 3001)
    for (l, m) in waveform.modes_from_mask(31):
        h = waveform.mode(src, l, m, t, 0.0)
        z = h * np.exp(1j * waveform.mode_phase(src, l, m, t)[0])
        assert np.max(np.abs(z.imag)) <= 1e-12 * np.max(np.abs(h))
        assert np.min(z.real) >= -1e-12 * np.max(np.abs(h))


@pytest.mark.parametrize("orbit,gen,nested,precessing", [
    ("rigid", 15, False, False), ("kepler", 20, False, False),
    ("kepler", 20, True, False), ("kepler", 20, False, True), ("rigid", 20, True, True)])
def test_point_response_matches_the_sampled_pipeline(orbit, gen, nested, precessing):
    """The continuous-time response against the independent Lagrange path.
    With the merger after the grid's end h is band-limited everywhere and the
    two agree to FP64 rounding: ~1e-12 rad of a ~1e4 rad phase, amplified by
    the cancellations of h(t_s) - h(t_r) and of TDI 2 to ~1e-9 of the output
    (the gap does not change between p = 7, 15 and 31).  (Within ~600 s of the grid's
    end, where this signal is cut off, the sampled path's stencils reach past
    the last sample and read zeros: outputs there are not compared.)"""
    s = _setup(precessing, orbit=orbit, tdi_gen=gen, tdi_nested=nested)
    th = _theta(precessing, tc=1.4 * DAY)
    idx = np.array([40, 700, 3000, 8000, 12000, 15000, 16500, 17000])
    ref = pipeline.aet(th, s, idx=idx)
    pt = H.point_aet(th, s, s.t0 + idx * s.dt).sum(axis=0)
    assert np.max(np.abs(pt.imag)) > 0.0                  # the quadrature is carried
    assert np.max(np.abs(pt.real - ref)) <= 5e-9 * np.max(np.abs(ref))


def test_point_response_near_a_merger_differs_only_by_the_stencil_error():
    """Near the stand-in's merger attachment (h only C1) the sampled path's
    interpolation error is large; away from it the two agree."""
    s = _setup()
    th = _theta()
    src = waveform.source(th, False)
    idx = np.array([2000, 6000, 10000, 16000])
    ref = pipeline.aet(th, s, idx=idx)
    pt = H.point_aet(th, s, s.t0 + idx * s.dt).sum(axis=0).real
    assert np.max(np.abs(pt - ref)) <= 5e-9 * np.max(np.abs(ref))
    near = np.array([int(src["tm"] / s.dt) + d for d in (-8, 0, 8)])
    ref = pipeline.aet(th, s, idx=near)
    pt = H.point_aet(th, s, s.t0 + near * s.dt).sum(axis=0).real
    assert np.max(np.abs(pt - ref)) <= 1e-3 * np.max(np.abs(ref))


@pytest.fixture(scope="module")
def aligned_day():
    s = _setup()
    th0 = _theta()
    x0 = H.continuous_aet(th0, s)
    th = _nearby(th0)
    return s, th0, x0, th, H.continuous_aet(th, s)


def test_the_fiducial_is_reproduced_exactly(aligned_day):
    s, th0, x0, _, _ = aligned_day
    nodes = wl.heterodyne_nodes(s.n, s.dt, th0[0], th0[1], th0[14])
    dz = H.node_deltas(th0, th0, s, nodes)
    assert np.all(dz == 0.0)
    m = H.model_aet(th0, th0, s, nodes, x0)
    assert np.array_equal(m, x0)
    d = x0 * 1.01
    assert H.loglike(th0, th0, s, d, nodes, x0) == likelihood.loglike(
        x0, d, s.dt, s.f_lo, s.f_hi, s.tdi_gen)


def test_a_node_at_every_sample_gives_the_continuous_response(aligned_day):
    s, th0, x0, th, full = aligned_day
    m = H.model_aet(th, th0, s, np.arange(s.n), x0)
    assert np.max(np.abs(m - full)) <= 1e-13 * np.max(np.abs(full))


def test_interpolation_error_is_fourth_order_in_the_node_spacing():
    """Inspiral only (merger after the grid): halving a uniform node spacing
    divides the model error by about sixteen (cubic interpolation; a linear one
    would divide it by four).  The last 1500 samples are left out: there the
    signal is cut off by the grid's end and terms whose delayed times leave the
    grid drop out, so the response is not smooth, and a cubic stencil reaches
    two node intervals beyond the sample it serves."""
    s = _setup(n=8640)
    th0 = _theta(tc=0.55 * DAY)
    th = _nearby(th0, 10.0)
    x0 = H.continuous_aet(th0, s)
    full = H.continuous_aet(th, s)
    err = []
    for step in (384, 192, 96):
        nodes = np.unique(np.r_[np.arange(0, s.n, step), s.n - 1])
        e = H.model_aet(th, th0, s, nodes, x0) - full
        err.append(np.max(np.abs(e[:, :-1500])))
    assert 9.0 <= err[0] / err[1] <= 24.0 and 9.0 <= err[1] / err[2] <= 24.0, err


def test_expansion_is_exact_for_cubic_envelopes_and_checks_its_nodes():
    """Step 5 on its own.  Node differences sampled from a complex cubic in the
    sample index expand to that cubic times the carrier at every sample, for
    any node spacing (wrong Lagrange weights fail this).  For a quartic the
    result is, sample by sample, numpy's degree-3 polyfit through the four
    nodes a .. a + 3, a = min(max(b - 1, 0), B - 4) around the sample's
    interval b (a shifted stencil fails this).  The node list is checked."""
    s = _setup(n=400)
    th0 = _theta()
    nodes = np.array([0, 3, 10, 11, 40, 100, 101, 250, 399])
    B = nodes.size
    rng = np.random.default_rng(4)
    coef = rng.normal(size=(5, 3, 5)) + 1j * rng.normal(size=(5, 3, 5))
    i = np.arange(s.n)
    c = H.carriers(th0, s, pipeline.grid(s))
    x0 = np.zeros((3, s.n))
    cubic = lambda x: sum(coef[..., k, None] * (x / 400.0) ** k for k in range(4))
    out = H.expand(cubic(nodes), th0, s, nodes, x0)
    want = np.stack([sum((c[j] * cubic(i)[j, ch]).real for j in range(5)) for ch in range(3)])
    assert np.max(np.abs(out - want)) <= 1e-12 * np.max(np.abs(want))
    quartic = lambda x: sum(coef[..., k, None] * (x / 400.0) ** k for k in range(5))
    zq = quartic(nodes)
    out = H.expand(zq, th0, s, nodes, x0)
    env = np.zeros((5, 3, s.n), dtype=complex)
    for k in range(s.n):
        b = min(np.searchsorted(nodes, k, side="right") - 1, B - 2)
        a = min(max(b - 1, 0), B - 4)
        xs = nodes[a:a + 4] / 400.0
        for j in range(5):
            for ch in range(3):
                env[j, ch, k] = (np.polyval(np.polyfit(xs, zq[j, ch, a:a + 4].real, 3), k / 400.0)
                                 + 1j * np.polyval(np.polyfit(xs, zq[j, ch, a:a + 4].imag, 3),
                                                   k / 400.0))
    want = np.stack([sum((c[j] * env[j, ch]).real for j in range(5)) for ch in range(3)])
    truth = np.stack([sum((c[j] * quartic(i)[j, ch]).real for j in range(5)) for ch in range(3)])
    assert np.max(np.abs(out - want)) <= 1e-9 * np.max(np.abs(want))
    assert np.max(np.abs(out - truth)) >= 1e-4 * np.max(np.abs(truth))   # not the quartic
    dz = np.zeros((5, 3, 4), dtype=complex)
    for bad in ([0, 5, 399], [1, 5, 9, 399], [0, 5, 9, 398], [0, 9, 5, 399]):
        with pytest.raises(ValueError):
            H.expand(dz[..., :len(bad)], th0, s, bad, x0)


def test_node_rule_reaches_the_continuous_likelihood(aligned_day):
    """The node rule at a posterior-width offset (SNR ~ 1.2e3): the heterodyned
    logL within 0.01 of the continuous-time logL, and a coarser rule errs
    more."""
    s, th0, x0, th, full = aligned_day
    ll = likelihood.loglike(full, x0, s.dt, s.f_lo, s.f_hi, s.tdi_gen)
    assert -200.0 < ll < -1.0
    errs = []
    for df in (2e-5, 5e-4):
        nodes = wl.heterodyne_nodes(s.n, s.dt, th0[0], th0[1], th0[14], df=df)
        errs.append(abs(H.loglike(th, th0, s, x0, nodes, x0) - ll))
    assert errs[0] <= 0.01 and errs[1] > errs[0], errs


def test_graded_spacing_keeps_a_walker_merging_outside_the_dense_window_accurate(aligned_day):
    """A walker merging 700 s after the fiducial (outside the dense window's
    520 s pad): with the raw rule its ringdown falls in the interval after the
    window, where the cubic through three dense nodes and one 12 h away
    amplifies the node values by ~1e6; with the graded spacing the logL stays
    within a few 1e-6 of the continuous one."""
    s, th0, x0, _, _ = aligned_day
    th = th0.copy()
    th[14] += 700.0
    ll = likelihood.loglike(H.continuous_aet(th, s), x0, s.dt, s.f_lo, s.f_hi, s.tdi_gen)
    err = [abs(H.loglike(th, th0, s, x0,
                         wl.heterodyne_nodes(s.n, s.dt, th0[0], th0[1], th0[14], grade=g), x0)
               - ll) / abs(ll) for g in (4.0, None)]
    assert err[0] <= 1e-5 and err[1] >= 1e-4, err


def test_node_rule_shape():
    th0 = _theta()
    n, dt = 1036800, 5.0
    nodes = wl.heterodyne_nodes(n, dt, th0[0], th0[1], 50.0 * DAY)
    d = np.diff(nodes)
    assert nodes[0] == 0 and nodes[-1] == n - 1 and np.all(d >= 1)
    assert np.max(d) <= 43200.0 / dt
    assert len(nodes) < 10000
    # every sample across the merger, sky delay included
    tc_i = int(50.0 * DAY / dt)
    assert np.all(d[(nodes[:-1] > tc_i - 104) & (nodes[:-1] < tc_i + 104)] == 1)
    # every 250 s over the start taper (the signal starts before the grid here)
    first = nodes[nodes * dt <= 1.0e4]
    assert first[0] == 0 and np.max(np.diff(first)) <= 50
    small = wl.heterodyne_nodes(100, dt, th0[0], th0[1], 1e9)
    assert small[0] == 0 and small[-1] == 99
    # adjacent spacings differ by at most the grading factor 4, so the cubic
    # through four nodes stays an interpolation of Lebesgue constant ~3
    # everywhere; the raw rule (a subset of the nodes) reaches ~1e3 and more
    # where the dense window meets a 12 h interval
    assert np.max(np.maximum(d[1:] / d[:-1], d[:-1] / d[1:])) <= 4.0
    raw = wl.heterodyne_nodes(n, dt, th0[0], th0[1], 50.0 * DAY, grade=None)
    assert np.all(np.isin(raw, nodes)) and nodes.size <= 1.05 * raw.size
    assert _lebesgue(nodes) <= 4.0 and _lebesgue(raw) >= 1e3


def _lebesgue(nodes):
    """max over samples of sum_q |w_q|: the cubic Lagrange weights of the
    expansion's stencil (nodes a .. a + 3, a = min(max(b - 1, 0), B - 4))."""
    B = nodes.size
    worst = 0.0
    for b in range(B - 1):
        a = min(max(b - 1, 0), B - 4)
        x = nodes[a:a + 4].astype(np.float64)
        for i in np.linspace(nodes[b], nodes[b + 1], 9):
            w = [np.prod([(i - x[t]) / (x[q] - x[t]) for t in range(4) if t != q])
                 for q in range(4)]
            worst = max(worst, float(np.sum(np.abs(w))))
    return worst
