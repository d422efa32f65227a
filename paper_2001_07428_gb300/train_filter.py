"""Train the filter network on plain runs of the method (GPU).

    python -m paper_2001_07428_gb300.train_filter [--runs 96,24,8] [--steps 6000] [--data PATH] [--out PATH]

With --data naming an existing file (default: the committed filter_runs.json) the plain runs are read
from it instead of being generated again.

1. Seeded plain runs (JTRLAN_MIXED_REORTH, no filter, residual 1e-7) on 8^4, 12^4 and 16^4 lattices
   with m0 ~ U[8, 10], kappa ~ U[0.1, 0.5], links from inputs.stencil_links: the lowest 101
   eigenvalues of each, and the spectral window from jtrlan_bounds (the network's inputs).
2. Samples: for each run and each nev in NEV_GRID, features -> Jackson-damped step coefficients with
   the cut between lambda_nev and lambda_{nev+1} (the library's jtrlan_damped_step kernel).
3. Full-batch Adam in the library's kernels (jtrlan_mlp_train); every 8th run is held out.
4. Writes the parameters and a summary (losses, held-out cut errors) to filter_mlp.npz.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

from . import inputs
from . import learned_filter as LF
from .solver import JTRLan

LATTICES = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16)]
NEV_TRUTH = 101


def run_record(i, dims, device="cuda"):
    """One plain run: (m0, kappa, sites, lo, hi, the lowest NEV_TRUTH eigenvalues)."""
    rng = np.random.default_rng(1000 + i)
    m0 = float(rng.uniform(8.0, 10.0))
    kappa = float(rng.uniform(0.1, 0.5))
    U, W = inputs.stencil_links(dims, 1000 + i)
    lo, hi = LF.stencil_bounds(U, W, dims, m0, kappa, device)
    s = JTRLan(kind="stencil", dims=dims, m0=m0, kappa=kappa, U=U, W=W, nev=NEV_TRUTH, m=220, mwin=100,
               tol=1e-7, precision="mixed_reorth", device=device)
    s.solve()
    ev, _, _ = s.pairs()
    s.close()
    return dict(i=i, dims=list(dims), m0=m0, kappa=kappa, sites=int(np.prod(dims)), lo=lo, hi=hi, ev=ev.tolist())


def samples(records, device="cuda"):
    X, taus, groups = [], [], []
    for r in records:
        a, b = LF.window(r["lo"], r["hi"])
        for nev in LF.NEV_GRID:
            X.append(LF.features(r["lo"], r["hi"], r["m0"], r["kappa"], nev, r["sites"]))
            taus.append(LF.cut_tau(np.asarray(r["ev"]), nev, a, b))
            groups.append(r["i"])
    taus = np.asarray(taus)
    return np.stack(X), LF.damped_targets(taus, device), taus, np.asarray(groups)


def tau_of(coeffs):
    """The cut encoded by a damped step: g_0 = c_0 = (pi - acos tau)/pi (j_0 = 1)."""
    return np.cos(np.pi * (1.0 - np.asarray(coeffs)[..., 0]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--runs", default="96,24,8", help="runs per lattice (8^4, 12^4, 16^4)")
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--data", default=LF.RUNS, help="cached plain-run records (json); generated if missing")
    ap.add_argument("--out", default=LF.WEIGHTS)
    args = ap.parse_args()
    counts = [int(c) for c in args.runs.split(",")]
    t0 = time.perf_counter()
    records = []
    if args.data and os.path.exists(args.data):
        records = json.load(open(args.data))
    else:
        i = 0
        for dims, cnt in zip(LATTICES, counts):
            for _ in range(cnt):
                records.append(run_record(i, dims))
                i += 1
        if args.data:
            json.dump(records, open(args.data, "w"))
    t_data = time.perf_counter() - t0
    X, T, taus, groups = samples(records)
    val = np.array([r["i"] % 8 == 7 for r in records])
    val_ids = {r["i"] for r, v in zip(records, val) if v}
    is_val = np.array([g in val_ids for g in groups])
    net = LF.FilterNet(seed=0)
    t1 = time.perf_counter()
    hist = []
    for steps, lr in ((args.steps // 2, 1e-3), (args.steps // 4, 3e-4), (args.steps - args.steps // 2 - args.steps // 4, 1e-4)):
        hist.append(net.train(X[~is_val], T[~is_val], steps, lr))
    t_train = time.perf_counter() - t1
    hist = np.concatenate(hist)
    pred = net.predict(X)
    dtau = np.abs(tau_of(pred) - taus)
    summary = dict(runs=len(records), samples=int(len(X)), train_samples=int((~is_val).sum()),
                   val_samples=int(is_val.sum()), steps=args.steps, loss_first=float(hist[0]),
                   loss_last=float(hist[-1]), val_loss=float(net.loss(X[is_val], T[is_val])),
                   val_tau_err_median=float(np.median(dtau[is_val])), val_tau_err_max=float(dtau[is_val].max()),
                   train_tau_err_median=float(np.median(dtau[~is_val])), data_seconds=t_data,
                   train_seconds=t_train, lattices=[list(d) for d in LATTICES], runs_per_lattice=counts,
                   degree=LF.DEGREE)
    net.save(args.out, **summary)
    print(json.dumps(summary), flush=True)


if __name__ == "__main__":
    main()
