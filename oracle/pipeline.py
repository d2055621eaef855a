"""One walker end to end: parameters -> h+, hx -> y_slr -> X,Y,Z -> A,E,T
-> logL (Sec. II.A - II.B), FP64.

``Setup`` mirrors the per-run configuration (grid, band, TDI generation and
delay form, channel mask, Lagrange order, orbit model, mode mask, precessing
flag).
"""
from dataclasses import dataclass

import numpy as np

from . import likelihood, response, waveform


@dataclass(frozen=True)
class Setup:
    dt: float = 5.0
    n: int = 17280
    t0: float = 0.0
    f_lo: float = 1e-4
    f_hi: float = 0.02
    tdi_gen: int = 15
    channel_mask: int = 7
    lagrange_order: int = 31
    orbit: object = "rigid"       # "rigid" | "kepler" | an orbits.OrbitTable
    mode_mask: int = 1            # bit0 (2,2) .. bit4 (4,4)
    precessing: bool = False
    tdi_nested: bool = False      # TDI delays as nested operator products


def grid(s: Setup, n=None):
    n = s.n if n is None else n
    return s.t0 + np.arange(n) * s.dt


def polarizations(theta, s: Setup, n=None):
    return waveform.plus_cross(theta, grid(s, n), s.t0, s.mode_mask, s.precessing)


def links(theta, s: Setup, n=None, idx=None):
    hp, hc = polarizations(theta, s, n)
    return response.all_links(hp, hc, s.t0, s.dt, s.orbit, theta[11], theta[12],
                              s.lagrange_order, idx)


def aet(theta, s: Setup, n=None, idx=None):
    """A, E, T on the whole grid, or at output indices ``idx`` (sparse: y is
    computed only where the TDI stencils read it)."""
    n = s.n if n is None else n
    hp, hc = polarizations(theta, s, n)
    if idx is None:
        y = response.all_links(hp, hc, s.t0, s.dt, s.orbit, theta[11], theta[12],
                               s.lagrange_order)
    else:
        need = response.tdi_support(idx, n, s.dt, s.orbit, s.tdi_gen,
                                    s.lagrange_order, s.t0, s.tdi_nested)
        part = response.all_links(hp, hc, s.t0, s.dt, s.orbit, theta[11], theta[12],
                                  s.lagrange_order, need)
        y = {}
        for l, vals in part.items():
            full = np.zeros(n)
            full[need] = vals
            y[l] = full
    X, Y, Z = response.tdi_xyz(y, n, s.t0, s.dt, s.orbit, s.tdi_gen,
                               s.lagrange_order, idx, s.tdi_nested)
    return np.stack(response.aet_from_xyz(X, Y, Z))


def loglike(theta, s: Setup, data_aet, n=None):
    h = aet(theta, s, n)
    return likelihood.loglike(h, data_aet, s.dt, s.f_lo, s.f_hi, s.tdi_gen,
                              s.channel_mask)
