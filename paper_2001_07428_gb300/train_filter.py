"""Train the filter network on plain runs of the method (GPU).

    python -m paper_2001_07428_gb300.train_filter [--runs 1000,1000,8] [--steps 6000] [--data PATH] [--out PATH]
                                                  [--generate] [--concurrency P] [--tol 1e-7]

With --data naming an existing file (default: the committed filter_runs.json) the plain runs are read
from it; --generate runs them again and writes that file.

1. Seeded plain runs (JTRLAN_MIXED_REORTH, no filter) on 8^4 and 12^4 lattices (and a few 16^4 runs
   that cover the smallest nev/sites fractions) with m0 ~ U[8, 10], kappa ~ U[0.1, 0.5], links from
   inputs.stencil_links, run i seeded with 1000 + i: the lowest 101 eigenvalues of each, and the
   spectral window from jtrlan_bounds (the network's inputs).  With --concurrency P, P runs proceed at
   once, each on its own CUDA stream and context (small lattices leave most of the GPU idle); these
   runs use the separate-launch Gram-Schmidt and the CUDA-core rotation, so that no cooperative or
   tensor-memory kernel of one run waits for resources another run holds.
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

import ctypes

import numpy as np
import torch

from . import binding as B
from . import inputs
from . import learned_filter as LF
from .solver import JTRLan

LATTICES = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16)]
NEV_TRUTH = 101


def run_record(i, dims, device="cuda", tol=1e-7, isolated=False):
    """One plain run: (m0, kappa, sites, lo, hi, the lowest NEV_TRUTH eigenvalues)."""
    rng = np.random.default_rng(1000 + i)
    m0 = float(rng.uniform(8.0, 10.0))
    kappa = float(rng.uniform(0.1, 0.5))
    U, W = inputs.stencil_links(dims, 1000 + i)
    t0 = time.perf_counter()
    lo, hi = LF.stencil_bounds(U, W, dims, m0, kappa, device)
    s = JTRLan(kind="stencil", dims=dims, m0=m0, kappa=kappa, U=U, W=W, nev=NEV_TRUTH, m=220, mwin=100,
               tol=tol, precision="mixed_reorth", gs_split=isolated, rotate_simt=isolated, device=device)
    st = s.solve()
    ev = np.zeros(NEV_TRUTH)
    B.jtrlan_pairs(s.ctx, 0, ev.ctypes.data_as(ctypes.c_void_p), None, None)
    s.close()
    return dict(i=i, dims=list(dims), m0=m0, kappa=kappa, sites=int(np.prod(dims)), lo=lo, hi=hi, ev=ev.tolist(),
                tol=tol, n_matvec=int(st["n_matvec"]), seconds=round(time.perf_counter() - t0, 3))


def generate(plan, device="cuda", tol=1e-7, concurrency=1, log=None):
    """Runs the plain runs of `plan` (a list of (i, dims)); with concurrency > 1, that many at once,
    each in a host thread with its own CUDA stream (the library releases the interpreter lock in its
    calls, and each context enqueues on the stream current at its creation)."""
    if concurrency <= 1:
        out = []
        for i, dims in plan:
            out.append(run_record(i, dims, device, tol))
            if log:
                log(out[-1])
        return out
    import concurrent.futures as cf
    import threading
    local = threading.local()

    def work(item):
        i, dims = item
        if not hasattr(local, "stream"):
            local.stream = torch.cuda.Stream(device=device)
        with torch.cuda.stream(local.stream):
            r = run_record(i, dims, device, tol, isolated=True)
        if log:
            log(r)
        return r

    with cf.ThreadPoolExecutor(max_workers=concurrency) as ex:
        return sorted(ex.map(work, plan), key=lambda r: r["i"])


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
    ap.add_argument("--runs", default="1000,1000,8", help="runs per lattice (8^4, 12^4, 16^4)")
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--data", default=LF.RUNS, help="plain-run records (json)")
    ap.add_argument("--generate", action="store_true", help="run the plain runs again and write --data")
    ap.add_argument("--concurrency", type=int, default=1)
    ap.add_argument("--tol", type=float, default=1e-7)
    ap.add_argument("--out", default=LF.WEIGHTS)
    ap.add_argument("--add", default=None, help="LxLxLxL:COUNT -- run COUNT more runs on that lattice and append them")
    args = ap.parse_args()
    counts = [int(c) for c in args.runs.split(",")]
    t0 = time.perf_counter()
    if args.generate or not os.path.exists(args.data):
        plan, i = [], 0
        for dims, cnt in zip(LATTICES, counts):
            plan += [(i + k, dims) for k in range(cnt)]
            i += cnt
        records = generate(plan, tol=args.tol, concurrency=args.concurrency,
                           log=lambda r: print(json.dumps({k: r[k] for k in ("i", "dims", "seconds", "n_matvec")}),
                                               flush=True))
        json.dump(records, open(args.data, "w"))
    else:
        records = json.load(open(args.data))
    if args.add:
        lat, cnt = args.add.split(":")
        dims = tuple(int(v) for v in lat.split("x"))
        start = max(r["i"] for r in records) + 1
        plan = [(start + k, dims) for k in range(int(cnt))]
        records += generate(plan, tol=args.tol, concurrency=args.concurrency,
                            log=lambda r: print(json.dumps({k: r[k] for k in ("i", "dims", "seconds", "n_matvec")}),
                                                flush=True))
        json.dump(records, open(args.data, "w"))
    t_data = time.perf_counter() - t0
    counts = [sum(1 for r in records if tuple(r["dims"]) == tuple(d)) for d in LATTICES]
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
