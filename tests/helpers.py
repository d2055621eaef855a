"""Shared test helpers: oracle setups mirroring a GPU config, and error norms."""
import numpy as np

from oracle import pipeline

ORBIT_NAMES = {0: "rigid", 1: "kepler"}


def oracle_setup(cfg):
    """oracle.pipeline.Setup for a workloads config dict."""
    return pipeline.Setup(dt=cfg["dt"], n=cfg["n"], t0=cfg["t0"], f_lo=cfg["f_lo"],
                          f_hi=cfg["f_hi"], tdi_gen=cfg["tdi_gen"],
                          channel_mask=cfg["channel_mask"],
                          lagrange_order=cfg["lagrange_order"],
                          orbit=ORBIT_NAMES[cfg["orbit"]], mode_mask=cfg["mode_mask"],
                          precessing=bool(cfg["precessing"]),
                          tdi_nested=bool(cfg.get("tdi_nested", 0)))


def gpu_kwargs(cfg):
    return dict(dt=cfg["dt"], n=cfg["n"], t0=cfg["t0"], f_lo=cfg["f_lo"], f_hi=cfg["f_hi"],
                tdi_gen=cfg["tdi_gen"], channel_mask=cfg["channel_mask"],
                lagrange_order=cfg["lagrange_order"], orbit=cfg["orbit"],
                mode_mask=cfg["mode_mask"], precessing=cfg["precessing"],
                tdi_nested=cfg.get("tdi_nested", 0))


def norm_rel(got, want):
    """max |got - want| / max |want| (the norm-relative error of a series)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = np.max(np.abs(want))
    if scale == 0.0:
        return float(np.max(np.abs(got)))
    return float(np.max(np.abs(got - want)) / scale)
