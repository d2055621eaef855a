"""Throughput sweep of the batched likelihood (walker count x duration x
spin model x orbit x precision), printed as a markdown table.

    python -m paper_2501_08261_gb300.sweep [--quick]

Each point creates a context, injects the first walker's response as
zero-noise data, autotunes the launch shapes (lisa_td_autotune), runs 2
warm-up and 3 timed lisa_td_loglike_batch calls with
the library's stage timing on, and reports logL evals/s, walker-samples/s and
the share of the two largest stages.  Inputs are the seeded prior draws of
workloads.prior_draws.
"""
import argparse
import itertools
import json

import numpy as np

from . import api, workloads

DAYS = {1: 17280, 7: 120960, 30: 518400, 60: 1036800}


def point(W, days, precessing, orbit, precision, steps=3, warmup=2):
    import torch
    cfg = workloads.config("c2_hm_60d", n=DAYS[days], orbit=orbit, precessing=int(precessing),
                           tdi_gen=20)
    kw = {k: cfg[k] for k in ("dt", "n", "t0", "f_lo", "f_hi", "tdi_gen", "channel_mask",
                              "lagrange_order", "orbit", "mode_mask", "precessing")}
    th = workloads.prior_draws(W, cfg["n"], cfg["dt"], seed=6, precessing=precessing)
    lk = api.Likelihood(precision=precision, max_walkers=W, **kw)
    p = torch.as_tensor(th, device="cuda")
    d = lk.tdi(lk.project(p[:1]))[:, :, 0].to(torch.float64).contiguous()
    lk.set_data(d)
    api.lisa_td_autotune(lk.ctx, p, W)          # launch shapes for this point
    out = torch.empty(W, dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        api.lisa_td_loglike_batch(lk.ctx, p, W, out)
    torch.cuda.synchronize()
    api.lisa_td_profile(lk.ctx, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        api.lisa_td_loglike_batch(lk.ctx, p, W, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    stages, calls = api.lisa_td_profile_read(lk.ctx)
    lk.close()
    tot = sum(stages.values())
    top = sorted(stages.items(), key=lambda kv: -kv[1])[:2]
    return {"W": W, "days": days, "spins": "precessing" if precessing else "aligned",
            "orbit": {0: "rigid", 1: "Keplerian"}[orbit], "precision": ("FP64", "mixed")[precision],
            "ms_per_step": round(ms, 3), "evals_per_s": round(W / (ms * 1e-3), 2),
            "walker_samples_per_s": W * cfg["n"] / (ms * 1e-3),
            "top_stages": [(k, round(100 * v / tot, 1)) for k, v in top]}


def grid(quick=False):
    Ws = (1, 16, 64, 256) if quick else (1, 16, 64, 256, 1024)
    pts = []
    for W, days, prec in itertools.product(Ws, (1, 7, 30, 60), (False, True)):
        pts.append((W, days, prec, 1, 1))                       # mixed, Keplerian
    for W in Ws:
        pts.append((W, 60, False, 0, 1))                         # mixed, rigid equal-arm
    for W, days in itertools.product((1, 16, 64), (1, 7)):
        pts.append((W, days, False, 1, 0))                       # FP64 path
    return pts


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--json", default=None, help="also write the points to this file")
    args = ap.parse_args()
    from . import build
    build.build()
    rows = [point(*p) for p in grid(args.quick)]
    print("| walkers | days | spins | orbit | precision | ms / step | logL evals/s | "
          "walker-samples/s | largest stages |")
    print("|---:|---:|---|---|---|---:|---:|---:|---|")
    for r in rows:
        print(f"| {r['W']} | {r['days']} | {r['spins']} | {r['orbit']} | {r['precision']} | "
              f"{r['ms_per_step']:.2f} | {r['evals_per_s']:.1f} | {r['walker_samples_per_s']:.3e} | "
              + ", ".join(f"{k} {v}%" for k, v in r["top_stages"]) + " |")
    if args.json:
        with open(args.json, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
