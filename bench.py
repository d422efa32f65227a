"""Benchmark: time to 100 eigenpairs at residual <= 1e-8 on the 24^3 x 48 stencil, learned-filter form.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference] [--workload NAME]

Default workload: the 24^3 x 48 periodic stencil (n = 3,981,312, complex64 links, m0 8.5, kappa 0.3,
seed 1), nev 100, m 200, mwin 100, tol 1e-8.  One "step" is one whole time to solution of the chosen
form, with the operator already resident in HBM:
  jtrlan_bounds on the solver's context (30 Lanczos steps) -> features -> the filter network's
  inference (library kernels) -> jtrlan_set_filter -> jtrlan_solve (Algorithm 1 on B = p(A) in
  JTRLAN_MIXED_REORTH: compensated-FP32 products and Gram-Schmidt on a (hi, lo) basis, tensor-core
  restart rotation, FP64 alpha/beta, Ritz solve and residuals; every pair certified by A's residual).

* value: mean device time per step over the K timed steps (CUDA events on the library stream; L2
  flushed before every step, outside the events), max over ranks.
* vs_plain_fp64: one plain FP64 J-TRLan solve of the same workload on the same GPU (same complex64
  links), its time, and the relative difference of every one of the 100 eigenvalues.
* stencil_fp32: the FP32 stencil matvec's GB/s on this lattice against the measured HBM peak.
* roofline: the kernel class with the largest device time in one extra profiled step (per-launch
  CUDA events inside the library), its algorithmic work over its summed time.
* e2e: the same step through the C ABI from pinned HOST buffers -- jtrlan_create (H2D of the links),
  bounds, inference, set_filter, solve, jtrlan_pairs into pinned host memory (D2H of the eigenvectors),
  destroy.
* cpu_baseline: the CPU FP64 oracle timed on a bounded sample of the same workload (its stencil product,
  single Lanczos steps, a slice of the restart rotation), projected to a whole plain-FP64 solve with
  the operation counts of the plain FP64 GPU solve; single-threaded and with BLAS on all host cores.
* --impl reference: the oracle itself is the reference arm (there is no reference code): each step is
  one Lanczos step (Algorithm 2) of the oracle at full size, timed as measured.
--workload stencil_8x8x8x8 runs the 8^4 suite instead (plain FP64 headline, both mixed forms, invert
mode, the 16^4 comparison, rotation and stencil rooflines, the batched dense instances).
Under torchrun with N > 1 every rank solves its own replica (the path has no exchange step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2001_07428_gb300 import inputs  # noqa: E402

GOLDEN = os.path.join(ROOT, "tests", "golden")
TOL = 1e-8
FP64_PEAK_DERIVED = 152 * 2 * 2 * 2.07e9 / 1e12   # SMs x DFMA/clk/SM x flop/FMA x max clock


def fp64_peak_tflops(peaks=None):
    """The FP64 FMA peak: measured by the library's FMA loop when `peaks` holds it, else derived."""
    if peaks and peaks.get("fp64_fma_tflops"):
        return peaks["fp64_fma_tflops"], "measured: FP64 FMA loop (jtrlan_measure_peaks)"
    return FP64_PEAK_DERIVED, "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"
L2_FLUSH_BYTES = 512 << 20


class L2Flush:
    """Flushes L2 between timed runs: writes one 512 MB buffer (the workload's data leaves L2), then
    reads a second 512 MB buffer, so that the write's dirty lines are written back here and not inside
    the next timed region (L2 is left holding clean, unrelated lines)."""

    def __init__(self, torch, dev):
        self.a = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        self.b = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def __call__(self):
        self.a.zero_()
        self.b.amax()

# Algorithmic cost per unit of work (see the library's jtrlan_profile documentation).
#   matvec / resid: per lattice site, 32 complex 3x3 matrix-vector products (9 complex FMA each,
#     8 flop) = 2304 flop; bytes = 84 complex words (72 link + 6 in + 6 out) x 16 B (c128).
#   gs_first / gs_dot / gs_update: per row pair x column, 4 complex FMA = 32 flop; bytes = the two
#     complex128 basis entries read = 32 B.
#   rotate: per real multiply-add 2 flop; bytes negligible per unit (V read once, counted apart).
FLOP_PER_UNIT = {"matvec": 2304.0, "resid": 2304.0, "gs_first": 32.0, "gs_dot": 32.0, "gs_update": 32.0,
                 "gs_step": 32.0, "rotate": 1.0}
BYTES_PER_UNIT = {"matvec": 84 * 16.0, "resid": 84 * 16.0, "gs_first": 32.0, "gs_dot": 32.0,
                  "gs_update": 32.0, "gs_step": 32.0}


# DRAM bytes (read + write) per launch from one ncu capture of a kernel class's dominant kernel, with the
# SHA-256 of the source file the capture was built from: the figure is reported only while that file
# is unchanged (roofline.traffic is null otherwise).
NCU_TRAFFIC = {
    "matvec": dict(bytes=688.2e6, workload="stencil_24x24x24x48", kernel="stencil_df_cheb_kernel<float2> (middle step)",
                   source="paper_2001_07428_gb300/csrc/gsdf.cu",
                   sha256="f57efe4d702152935a4c602a1878b2d051606c3f149bf54843bd0f03d7e79d1e"),
    "gs_step": dict(bytes=13.66e6, workload="stencil_8x8x8x8", kernel="gs_step_coop_kernel<double>",
                    source="paper_2001_07428_gb300/csrc/gs.cu",
                    sha256="25f4b188216fe6b311d90026b3e55046646e3a430ba0d7a2b9d8b809fdae98b5"),
}


def source_sha(rel):
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def ncu_traffic(kind, workload_name):
    t = NCU_TRAFFIC.get(kind)
    if not t or t["workload"] != workload_name or source_sha(t["source"]) != t["sha256"]:
        return None
    return t["bytes"]


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def workload(name):
    w = dict(inputs.WORKLOADS[name])
    if w["kind"] != "stencil":
        raise SystemExit("bench.py times the stencil workloads")
    return w


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- ranks (replicas: no collective on the data path)
def max_over_ranks(value, world, device):
    """The largest `value` over the ranks: every rank runs the same solve on its own GPU, and the job
    is as slow as its slowest replica.  `device` holds the collective's tensor (cuda under NCCL, cpu
    under gloo)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks during the timed region
class Clocks:
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index):
        self.proc = None
        self.path = os.path.join("/tmp", f"jtrlan_clocks_{os.getpid()}.csv")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle sample
def oracle_sample(name, restarts):
    """Runs the oracle's Algorithm 1 for `restarts` outer iterations; returns (seconds, products A v)."""
    from oracle import jsym
    from oracle import trlan_jsym as tj
    w = workload(name)
    dims = w["dims"]
    U, W = inputs.stencil_links(dims, w["seed"])
    n = 6 * inputs.lattice_volume(dims)
    count = [0]

    def mv(x):
        count[0] += 1
        return jsym.stencil_matvec(U, W, dims, w["m0"], w["kappa"], x)

    t0 = time.perf_counter()
    try:
        tj.trlan_jsym(mv, n, w["nev"], w["m"], w["mwin"], TOL, max_restarts=restarts)
    except tj.NoConvergenceError:
        pass
    return time.perf_counter() - t0, count[0]


def cpu_baseline(name, full_products, restarts=4):
    """The oracle timed single-threaded in a child process (BLAS pinned to one thread), on its first
    `restarts` outer iterations, scaled to a whole solve by the number of products A v."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", name, "--sample-restarts", str(restarts)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        return {"value": None, "error": r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    value = d["seconds"] * full_products / d["products"]
    return {"value": value, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": f"first {restarts} outer iterations of the same solve ({d['products']} of {full_products} "
                      f"products A v, {d['seconds']:.1f} s), scaled by the product count"}


# ---------------------------------------------------------------- the mixed form where it is quoted
def mixed_at_16(B, torch, stream, flush, profiled_ms=None):
    """One timed solve each of plain FP64 and the double-float mixed form on the 16^4 workload
    (n = 393,216, nev = 50, m = 120, mwin = 60), after one untimed warm-up solve of each; with
    `profiled_ms` (a function of a context returning per-kernel device times) also one profiled
    solve of each."""
    import ctypes
    w = inputs.WORKLOADS["stencil_16x16x16x16"]
    dims = w["dims"]
    dev = torch.device("cuda", torch.cuda.current_device())
    U, W = inputs.stencil_links(dims, w["seed"])
    Ud, Wd = torch.from_numpy(U).to(dev), torch.from_numpy(W).to(dev)
    op = B.stencil_operator(dims, w["m0"], w["kappa"], Ud.data_ptr(), Wd.data_ptr())
    out = {"workload": "stencil_16x16x16x16", "n": 6 * inputs.lattice_volume(dims), "nev": w["nev"], "m": w["m"],
           "mwin": w["mwin"], "tol": TOL}
    evs = {}
    for name, prec in (("fp64", B.JTRLAN_FP64), ("mixed_reorth", B.JTRLAN_MIXED_REORTH)):
        ctx = B.jtrlan_create(op, B.params(w["nev"], w["m"], w["mwin"], TOL, precision=prec), stream.cuda_stream)
        B.jtrlan_solve(ctx)
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = B.jtrlan_solve(ctx)
        e1.record(stream)
        torch.cuda.synchronize()
        ev = np.zeros(w["nev"])
        res = np.zeros(w["nev"])
        B.jtrlan_pairs(ctx, 0, ev.ctypes.data_as(ctypes.c_void_p), None, res.ctypes.data_as(ctypes.c_void_p))
        B.jtrlan_destroy(ctx)
        evs[name] = ev
        out[name] = {"value": e0.elapsed_time(e1) / 1e3, "unit": "s", "n_matvec": st["n_matvec"],
                     "n_restarts": st["n_restarts"], "max_residual": float(res.max())}
        if profiled_ms is not None:
            ctxp = B.jtrlan_create(op, B.params(w["nev"], w["m"], w["mwin"], TOL, precision=prec, profile=1),
                                   stream.cuda_stream)
            out[name]["kernels"] = profiled_ms(ctxp)
            B.jtrlan_destroy(ctxp)
    out["speedup_vs_fp64"] = round(out["fp64"]["value"] / out["mixed_reorth"]["value"], 3)
    out["max_rel_eig_diff_vs_fp64"] = float(np.max(np.abs(evs["mixed_reorth"] - evs["fp64"]) / np.abs(evs["fp64"])))
    return out


# ---------------------------------------------------------------- invert mode (Algorithm 1, CG inner solves)
def invert_compare(B, torch, stream, flush, op, w, t_normal, ev_normal, reps=3):
    """Algorithm 1's invert mode on the headline workload: the same nev smallest pairs through
    A^{-1} (conjugate gradients to 1e-12 per product), timed like the headline (one warm-up, then the
    mean of `reps` solves, L2 flushed before each), against the normal-mode FP64 solve; and the paper's
    invert-mode comparison of N_MV (A^{-1} applications) between TRLAN-JSYM and plain TRLAN, TRLAN run
    with nev, m and mwin doubled to find both members of every pair."""
    import ctypes
    nev, m, mwin = w["nev"], w["m"], w["mwin"]
    out = {"workload": "stencil_8x8x8x8", "nev": nev, "m": m, "mwin": mwin, "tol": TOL, "cg_tol": 1e-12}
    ctx = B.jtrlan_create(op, B.params(nev, m, mwin, TOL, invert=1), stream.cuda_stream)
    st = B.jtrlan_solve(ctx)
    ts = []
    for _ in range(reps):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = B.jtrlan_solve(ctx)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    ev = np.zeros(nev)
    res = np.zeros(nev)
    B.jtrlan_pairs(ctx, 0, ev.ctypes.data_as(ctypes.c_void_p), None, res.ctypes.data_as(ctypes.c_void_p))
    B.jtrlan_destroy(ctx)
    t = statistics.mean(ts)
    out["jsym"] = {"value": t, "unit": "s", "n_matvec_inverse": st["n_matvec"], "n_cg_iters": st["n_cg_iters"],
                   "n_matvec_inner": st["n_matvec_inner"], "n_restarts": st["n_restarts"],
                   "max_residual": float(res.max()),
                   "max_rel_eig_diff_vs_normal_mode": float(np.max(np.abs(ev - ev_normal) / np.abs(ev_normal))),
                   "normal_mode_s": t_normal, "ratio_to_normal_mode": round(t / t_normal, 3)}
    ctx = B.jtrlan_create(op, B.params(2 * nev, 2 * m, 2 * mwin, TOL, invert=1, plain_trlan=1), stream.cuda_stream)
    st2 = B.jtrlan_solve(ctx)
    B.jtrlan_destroy(ctx)
    out["plain_trlan"] = {"n_matvec_inverse": st2["n_matvec"], "n_cg_iters": st2["n_cg_iters"],
                          "n_restarts": st2["n_restarts"], "nev": 2 * nev, "m": 2 * m, "mwin": 2 * mwin}
    out["n_matvec_ratio_trlan_over_jsym"] = round(st2["n_matvec"] / st["n_matvec"], 3)
    return out


# ---------------------------------------------------------------- FP32 stencil matvec vs HBM
STENCIL_LATTICES = {"16x16x16x16": (16, 16, 16, 16), "24x24x24x48": (24, 24, 24, 48)}


def stencil_apply_roofline(dims, reps=20, seed=4):
    """Times jtrlan_apply of the FP32 operator (a mixed-precision context, complex64 links) on the
    seeded lattice `dims`: median device time over `reps` launches, L2 flushed before each, and the
    algorithmic 84 complex64 words per site (72 link + 6 in + 6 out) per launch over that time."""
    import torch

    from paper_2001_07428_gb300 import binding as B
    dev = torch.device("cuda", torch.cuda.current_device())
    U, W = inputs.stencil_links(dims, seed)
    vol = inputs.lattice_volume(dims)
    n = 6 * vol
    Ud = torch.from_numpy(U.astype(np.complex64)).to(dev)
    Wd = torch.from_numpy(W.astype(np.complex64)).to(dev)
    del U, W
    stream = torch.cuda.current_stream(dev)
    op = B.stencil_operator(dims, 8.5, 0.3, Ud.data_ptr(), Wd.data_ptr(), dtype=B.JTRLAN_C64)
    ctx = B.jtrlan_create(op, B.params(1, 2, 1, TOL, precision=B.JTRLAN_MIXED), stream.cuda_stream)
    x = torch.from_numpy(inputs.random_vector(n, seed).astype(np.complex64)).to(dev)
    y = torch.empty_like(x)
    flush = L2Flush(torch, dev)
    for _ in range(3):
        B.jtrlan_apply(ctx, x.data_ptr(), y.data_ptr())
    ts = []
    for _ in range(reps):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.jtrlan_apply(ctx, x.data_ptr(), y.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e-3)
    B.jtrlan_destroy(ctx)
    t = statistics.median(ts)
    hbm, src = measured_peaks()
    algo = 84 * 8 * vol
    gbs = algo / t / 1e9
    return {"lattice": list(dims), "us": round(t * 1e6, 2), "algorithmic_bytes": algo, "gbs": round(gbs, 1),
            "frac_of_hbm": round(gbs / hbm, 4), "hbm_peak_gbs": hbm, "peak_source": src}


# ---------------------------------------------------------------- restart rotation on the tensor cores
# (n, m, kk) of the lattices' mixed-precision solves: the rotation of the nev candidate Ritz vectors
ROTATE_SHAPES = {"8x8x8x8": (24576, 60, 20), "16x16x16x16": (393216, 120, 50), "24x24x24x48": (3981312, 200, 100)}


def bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p)).get("bf16_tflops", 1900.0)), "measured (burst)"
    return 1900.0, "fallback"


def rotate_roofline(shape, reps=5, seed=6):
    """Times jtrlan_rotate_df (V Z for a (hi, lo) basis V, n x m, and FP64 Z, m x kk) on the tensor
    cores (path 0) and on the CUDA cores (path 1): median of `reps` calls, L2 flushed before each.  A
    call also allocates and frees its scratch, computes the row exponents of V and splits Z (about
    0.1 ms of the small case).  The tensor-core figure counts the BF16 MMA work issued: 28 digit
    pairs x 2 x (2n rounded up to 128) x (m rounded up to 16) x (kk rounded up to 32)."""
    import torch

    from paper_2001_07428_gb300 import binding as B
    n, m, kk = shape
    dev = torch.device("cuda", torch.cuda.current_device())
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    x = torch.randn(m, n, 2, dtype=torch.float64, device=dev, generator=g) / math.sqrt(2 * n)
    hi = x.float()
    lo = (x - hi.double()).float()
    del x
    V = torch.stack([hi[..., 0], hi[..., 1], lo[..., 0], lo[..., 1]], dim=-1).contiguous()
    del hi, lo
    Z = np.linalg.qr(np.random.default_rng(seed).standard_normal((m, m)))[0][:, :kk]
    Zd = torch.from_numpy(np.ascontiguousarray(Z.T)).to(dev)
    out = [torch.empty(kk, n, dtype=torch.complex128, device=dev) for _ in range(2)]
    stream = torch.cuda.current_stream(dev)
    flush = L2Flush(torch, dev)
    res = {}
    for path in (0, 1):
        B.jtrlan_rotate_df(V.data_ptr(), n, m, Zd.data_ptr(), kk, out[path].data_ptr(), path, stream.cuda_stream)
        ts = []
        for _ in range(reps):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.jtrlan_rotate_df(V.data_ptr(), n, m, Zd.data_ptr(), kk, out[path].data_ptr(), path, stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        res[path] = statistics.median(ts)
    diff = (out[0] - out[1]).abs().max().item()
    del V, out
    torch.cuda.empty_cache()
    peak, src = bf16_peak()
    mma = 28 * 2 * (-(-2 * n // 128) * 128) * (-(-m // 16) * 16) * (-(-kk // 32) * 32)
    algo = 2 * (2 * n) * m * kk
    tf = mma / res[0] / 1e12
    return {"n": n, "m": m, "kk": kk, "tensor_ms": round(res[0] * 1e3, 3), "cuda_core_ms": round(res[1] * 1e3, 3),
            "speedup": round(res[1] / res[0], 2), "max_abs_diff_between_paths": diff,
            "roofline": {"bound": "tensor", "achieved": round(tf, 1), "peak": peak, "unit": "TFLOP/s",
                         "frac": round(tf / peak, 4), "peak_source": src,
                         "work": "BF16 MMA flops issued (28 digit pairs)"},
            "fp64_equivalent_tflops": round(algo / res[0] / 1e12, 3)}


# ---------------------------------------------------------------- learned polynomial filter
LEARNED_LATTICES = {"16x16x16x16": dict(dims=(16, 16, 16, 16), nev=50, m=120, mwin=60),
                    "24x24x24x48": dict(dims=(24, 24, 24, 48), nev=100, m=200, mwin=100)}


def learned_compare(B, torch, lattice, with_fp64=False, seed=1, m0=8.5, kappa=0.3):
    """Time to nev pairs at residual 1e-8 on the seeded stencil (complex64 links, as the workload states):
    the learned-filter form (jtrlan_bounds + network inference + JTRLAN_MIXED_REORTH on B = p(A), every
    pair certified by A's true residual) against the same solver unfiltered and, optionally, plain FP64.
    Operator upload excluded; CUDA-synchronised wall clock around the solve calls."""
    from paper_2001_07428_gb300 import learned_filter as LF
    from paper_2001_07428_gb300.solver import JTRLan
    cfg = LEARNED_LATTICES[lattice]
    dims, nev, m, mwin = cfg["dims"], cfg["nev"], cfg["m"], cfg["mwin"]
    U, W = inputs.stencil_links(dims, seed)
    U, W = U.astype(np.complex64), W.astype(np.complex64)
    dev = "cuda:%d" % torch.cuda.current_device()
    kw = dict(kind="stencil", dims=dims, m0=m0, kappa=kappa, U=U, W=W, nev=nev, m=m, mwin=mwin, tol=TOL,
              links_dtype="c64", device=dev)
    out = {"workload": f"stencil_{lattice}", "n": 6 * inputs.lattice_volume(dims), "nev": nev, "m": m, "mwin": mwin,
           "tol": TOL, "links": "complex64"}
    net = LF.FilterNet.load(device=dev)

    def timed_solve(s):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = s.solve()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, st

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g, win, feat = LF.learned_filter(net, U, W, dims, m0, kappa, nev, device=dev)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    s = JTRLan(precision="mixed_reorth", filter_final_coeffs=g, filter_window=win, **kw)
    t, st = timed_solve(s)
    ev_l, _, res_l = s.pairs()
    s.close()
    # one more solve with the library's per-launch CUDA-event profile: where the learned form spends its time
    sp = JTRLan(precision="mixed_reorth", filter_final_coeffs=g, filter_window=win, profile=True, **kw)
    sp.solve()
    prof = sp.profile()
    sp.close()
    tot = sum(v["ms"] for v in prof.values()) or 1.0
    kernels = {k: {"ms": round(v["ms"], 2), "launches": v["launches"], "share": round(v["ms"] / tot, 4)}
               for k, v in prof.items() if v["launches"]}
    out["learned"] = {"value": t_setup + t, "unit": "s", "filter_setup_s": t_setup, "solve_s": t, "kernels": kernels,
                      "degree": len(g) - 1, "window": list(win), "cut_tau": float(np.cos(np.pi * (1 - g[0]))),
                      "n_matvec": st["n_matvec"], "n_resid_matvec": st["n_resid_matvec"],
                      "n_restarts": st["n_restarts"], "max_residual": float(res_l.max())}
    forms = [("mixed_reorth", "mixed_reorth")] + ([("fp64", "fp64")] if with_fp64 else [])
    for name, prec in forms:
        s = JTRLan(precision=prec, **kw)
        t, st = timed_solve(s)
        ev, _, res = s.pairs()
        s.close()
        out[name] = {"value": t, "unit": "s", "n_matvec": st["n_matvec"], "n_restarts": st["n_restarts"],
                     "max_residual": float(res.max())}
        out["learned"]["max_rel_eig_diff_vs_" + name] = float(np.max(np.abs(ev_l - ev) / np.abs(ev)))
        out["learned"]["speedup_vs_" + name] = round(t / out["learned"]["value"], 3)
    return out


# ---------------------------------------------------------------- J-TRLan vs plain TRLAN (Sec. 4, Case A)
CASE_A_JSYM = [(5, 10, 50), (5, 10, 100), (5, 10, 150), (5, 10, 200),
               (10, 20, 50), (10, 20, 100), (10, 20, 150), (10, 20, 200)]


def case_a_sweep(B, torch, count=10, n=2000, tol=1e-13):
    """The parameter sweep of the paper's Case A table on `count` regenerated matrices (inputs.case_a,
    seeds 0..count-1): the largest nev pairs with TRLAN-JSYM at (nev, mwin, m) and with plain TRLAN
    (W removed) at the doubled parameters, plain FP64, tol 1e-13.  Reports [min, mean, max] of the
    outer iterations N_conv and of N_MV over the matrices, and the eigenvalue agreement with the
    generator's Lambda."""
    from paper_2001_07428_gb300.solver import JTRLan
    mats = [inputs.case_a(n, seed) for seed in range(count)]
    dev = "cuda:%d" % torch.cuda.current_device()
    rows = []
    for nev, mwin, m in CASE_A_JSYM:
        for name, (q, w, mm, plain) in (("TRLAN-JSYM", (nev, mwin, m, False)), ("TRLAN", (2 * nev, 2 * mwin, 2 * m, True))):
            nconv, nmv, err = [], [], 0.0
            for A11, A12, lam in mats:
                s = JTRLan(kind="dense", A11=A11, A12=A12, nev=q, m=mm, mwin=w, tol=tol, which="largest",
                           precision="fp64", plain_trlan=plain, device=dev)
                st = s.solve()
                ev, _, _ = s.pairs()
                s.close()
                top = np.sort(lam)[::-1][:nev]
                want = np.repeat(top, 2) if plain else top
                err = max(err, float(np.abs(ev - want).max()))
                nconv.append(st["n_restarts"])
                nmv.append(st["n_matvec"])
            rows.append({"algorithm": name, "nev": q, "mwin": w, "m": mm,
                         "N_conv": [int(min(nconv)), round(float(np.mean(nconv)), 1), int(max(nconv))],
                         "N_MV": [int(min(nmv)), round(float(np.mean(nmv)), 1), int(max(nmv))],
                         "max_abs_eig_err": err})
    return {"workload": f"case_a_n{n}_x{count}", "tol": tol, "which": "largest", "rows": rows}


# ---------------------------------------------------------------- batched dense instances
BATCH = dict(count=512, lo=64, hi=512, size_seed=2, seed0=1000, nev=8, m=24, mwin=12)


def batch_instances(count=None):
    """512 dense Hermitian J-symmetric instances (A11 = (G+G^H)/2, A12 = (K-K^T)/2, complex Gaussian),
    n uniform over the even numbers 64..512, seeded as the parity test seeds them (a smaller count
    takes the first instances of the same sequence, for profiling)."""
    count = count or BATCH["count"]
    sizes = inputs.batched_dense_sizes(count, BATCH["lo"], BATCH["hi"], seed=BATCH["size_seed"])
    return sizes, [inputs.dense_jsym(int(n) // 2, BATCH["seed0"] + i) for i, n in enumerate(sizes)]


def fp32_residual_floor(B, torch, stream, sizes, blocks, ops, picks=8):
    """Why the batch's reduced-precision form is compensated FP32, not FP32: for `picks` instances
    across the sizes, the converged FP64 eigenpairs (x, lambda) of the batch are evaluated with the
    library's FP32 product (jtrlan_apply of a context holding the FP32 operator) -- the residual
    ||A x - lambda x|| that FP32 arithmetic reports for pairs that are already accurate to 1e-8, next
    to the FP64 residual of the same pairs.  An FP32-arithmetic solve cannot certify below that floor."""
    import ctypes
    dev = torch.device("cuda", torch.cuda.current_device())
    nev = BATCH["nev"]
    order = np.argsort(sizes)
    idx = [int(order[k]) for k in np.linspace(0, len(sizes) - 1, picks).astype(int)]
    bt = B.jtrlan_batch_create([ops[i] for i in idx], B.params(nev, BATCH["m"], BATCH["mwin"], TOL), stream.cuda_stream)
    B.jtrlan_batch_solve(bt)
    ev = np.zeros((len(idx), nev))
    B.jtrlan_batch_results(bt, ev.ctypes.data_as(ctypes.c_void_p), None, None)
    rows = []
    for q, i in enumerate(idx):
        n = int(sizes[i])
        X = torch.empty((nev, n), dtype=torch.complex128, device=dev)
        B.jtrlan_batch_vectors(bt, q, ctypes.c_void_p(X.data_ptr()))
        ctx = B.jtrlan_create(ops[i], B.params(1, 2, 1, TOL, precision=B.JTRLAN_MIXED), stream.cuda_stream)
        r32, r64 = [], []
        A11, A12 = blocks[i]
        for c in range(nev):
            x = X[c]
            x32 = x.to(torch.complex64)
            y32 = torch.empty_like(x32)
            B.jtrlan_apply(ctx, x32.data_ptr(), y32.data_ptr())
            torch.cuda.synchronize()
            xh = x.cpu().numpy()
            r32.append(float(np.linalg.norm(y32.cpu().numpy().astype(np.complex128) - ev[q, c] * xh)))
            h = n // 2
            y64 = np.concatenate([A11 @ xh[:h] + A12 @ xh[h:], np.conj(A11) @ xh[h:] - np.conj(A12) @ xh[:h]])
            r64.append(float(np.linalg.norm(y64 - ev[q, c] * xh)))
        B.jtrlan_destroy(ctx)
        rows.append({"n": n, "max_residual_fp32_arithmetic": max(r32), "max_residual_fp64": max(r64)})
    B.jtrlan_batch_destroy(bt)
    return {"instances": rows, "tol": TOL,
            "min_fp32_floor": min(r["max_residual_fp32_arithmetic"] for r in rows),
            "note": "converged FP64 pairs evaluated with the FP32 product: FP32 arithmetic cannot reach 1e-8"}


def batched_oracle_sample(picks):
    """Oracle (CPU FP64) time for the instances `picks` of the batch; run as a subprocess."""
    from oracle import jsym
    from oracle import trlan_jsym as tj
    sizes, blocks = batch_instances()
    t0 = time.perf_counter()
    for i in picks:
        A11, A12 = blocks[i]
        tj.trlan_jsym(lambda x: jsym.dense_matvec(A11, A12, x), int(sizes[i]), BATCH["nev"], BATCH["m"],
                      BATCH["mwin"], TOL)
    return time.perf_counter() - t0


def batched_dense(B, torch, stream, steps, warmup, cpu=True, count=None, shape=None, forms=("fp64", "mixed_reorth"),
                  peaks=None):
    """The batch in one persistent launch per solve (CUDA-graph replay, autotuned launch shape), plain
    FP64 and the compensated-FP32 form; K timed solves each after W warm-up solves.  Inputs (408 MB of
    packed blocks) exceed L2.  Roofline: algorithmic matvec work (32 flop and 32 bytes per (row pair,
    column) of the packed blocks per product) over the solve time."""
    import ctypes
    sizes, blocks = batch_instances(count)
    count = len(sizes)
    dev = torch.device("cuda", torch.cuda.current_device())
    h2 = (sizes // 2).astype(np.int64) ** 2
    out = {"workload": f"dense_batch_{count}_n64-512", "count": count, "n_range": [BATCH["lo"], BATCH["hi"]],
           "nev": BATCH["nev"], "m": BATCH["m"], "mwin": BATCH["mwin"], "tol": TOL,
           "packed_bytes": int(2 * 16 * h2.sum())}
    Ad = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)) for a, b in blocks]
    ops = [B.dense_operator(2 * a.shape[0], a.data_ptr(), b.data_ptr()) for a, b in Ad]
    evs = {}
    hbm, hsrc = measured_peaks()
    precs = {"fp64": B.JTRLAN_FP64, "mixed_reorth": B.JTRLAN_MIXED_REORTH}
    for name in forms:
        prec = precs[name]
        bt = B.jtrlan_batch_create(ops, B.params(BATCH["nev"], BATCH["m"], BATCH["mwin"], TOL, precision=prec),
                                   stream.cuda_stream)
        if shape:
            B.jtrlan_batch_set_shape(bt, shape[0], shape[1])
            tuned = {"threads": shape[0], "ctas_per_sm": shape[1], "best_ms": None}
        else:
            tuned = B.jtrlan_batch_tune(bt)
        for _ in range(warmup):
            st = B.jtrlan_batch_solve(bt)
        ts = []
        for _ in range(steps):
            st = B.jtrlan_batch_solve(bt)
            ts.append(st["solve_ms"] * 1e-3)
        ev = np.zeros((count, BATCH["nev"]))
        res = np.zeros_like(ev)
        ist = np.zeros((count, B.BATCH_STATS), dtype=np.int32)
        B.jtrlan_batch_results(bt, ev.ctypes.data_as(ctypes.c_void_p), res.ctypes.data_as(ctypes.c_void_p),
                               ist.ctypes.data_as(ctypes.c_void_p))
        B.jtrlan_batch_destroy(bt)
        # one more solve with per-phase cycle counters (thread 0 of each CTA reads clock64 at barriers)
        bp = B.jtrlan_batch_create(ops, B.params(BATCH["nev"], BATCH["m"], BATCH["mwin"], TOL, precision=prec,
                                                 profile=1), stream.cuda_stream)
        B.jtrlan_batch_set_shape(bp, tuned["threads"], tuned["ctas_per_sm"])
        sp = B.jtrlan_batch_solve(bp)
        B.jtrlan_batch_destroy(bp)
        evs[name] = ev
        t = statistics.mean(ts)
        prods = (ist[:, 0] + ist[:, 3]).astype(np.int64)
        flop = float(32 * (prods * h2).sum())
        byts = float(2 * 16 * (prods * h2).sum())
        e = {"value": t, "unit": "s", "instances_per_s": round(count / t, 1), "n_ok": int(st["n_ok"]),
             "n_matvec": int(st["n_matvec"]), "n_resid_matvec": int(st["n_resid_matvec"]),
             "max_outer_iterations": int(st["max_restarts"]), "max_residual": float(res.max()),
             "grid": st["grid"], "threads": st["threads"], "tuned": tuned, "graph": st["graph"],
             "n_gs_passes": int(st["n_gs_passes"]), "n_ritz_fallbacks": int(st["n_ritz_fallbacks"]),
             "phase_share": {k: round(v, 4) for k, v in sp["phase_frac"].items()},
             "matvec_tflops": round(flop / t / 1e12, 4), "matvec_gbs": round(byts / t / 1e9, 1)}
        fp64_peak, fp64_src = fp64_peak_tflops(peaks)
        if name == "fp64":   # FP64-pipe-bound: the products' FP64 flops against the measured FP64 FMA peak
            e["bound"] = "alu (FP64 pipe)"
            e["frac_of_fp64_peak"] = round(e["matvec_tflops"] / fp64_peak, 4)
            e["fp64_peak_tflops"], e["fp64_peak_source"] = round(fp64_peak, 3), fp64_src
        else:                # compensated FP32: FP32-issue-bound; matvec_tflops counts FP64-equivalent flops
            e["bound"] = "alu (FP32 issue; compensated arithmetic)"
            e["matvec_tflops_fp64_equivalent"] = e.pop("matvec_tflops")
        e["frac_of_hbm"] = round(e["matvec_gbs"] / hbm, 4)
        out[name] = e
    if len(forms) == 2:
        out["speedup_vs_fp64"] = round(out["fp64"]["value"] / out["mixed_reorth"]["value"], 3)
        out["max_rel_eig_diff_vs_fp64"] = float(np.max(np.abs(evs["mixed_reorth"] - evs["fp64"]) / np.abs(evs["fp64"])))
    out["hbm_peak_gbs"], out["hbm_peak_source"] = hbm, hsrc
    out["fp32_residual_floor"] = fp32_residual_floor(B, torch, stream, sizes, blocks, ops)
    if count != BATCH["count"]:
        return out
    # end to end: pinned host blocks -> create (H2D) -> solve -> eigenvalues and vectors to host
    Hh = [(torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory()) for a, b in blocks]
    ops_h = [B.dense_operator(2 * a.shape[0], a.data_ptr(), b.data_ptr()) for a, b in Hh]
    Xh = torch.empty(int(sizes.sum()) * BATCH["nev"], dtype=torch.complex128).pin_memory()
    ev = np.zeros((count, BATCH["nev"]))
    chosen = min(forms, key=lambda k: out[k]["value"])
    prec = B.JTRLAN_FP64 if chosen == "fp64" else B.JTRLAN_MIXED_REORTH
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bt = B.jtrlan_batch_create(ops_h, B.params(BATCH["nev"], BATCH["m"], BATCH["mwin"], TOL, precision=prec),
                               stream.cuda_stream)
    B.jtrlan_batch_set_shape(bt, out[chosen]["tuned"]["threads"], out[chosen]["tuned"]["ctas_per_sm"])
    B.jtrlan_batch_solve(bt)
    B.jtrlan_batch_results(bt, ev.ctypes.data_as(ctypes.c_void_p), None, None)
    off = 0
    for i, n in enumerate(sizes):
        B.jtrlan_batch_vectors(bt, i, ctypes.c_void_p(Xh.data_ptr() + 16 * off))
        off += int(n) * BATCH["nev"]
    B.jtrlan_batch_destroy(bt)
    te = time.perf_counter() - t0
    out["e2e"] = {"form": chosen, "value": te, "unit": "s", "h2d_bytes": out["packed_bytes"],
                  "d2h_bytes": int(Xh.numel() * 16 + ev.size * 8)}
    if cpu:
        order = np.argsort(sizes)
        picks = [int(order[j]) for j in range(0, BATCH["count"], 16)]   # 32 instances across the sizes
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--batched-oracle-sample",
                            ",".join(map(str, picks))], capture_output=True, text=True, timeout=1800,
                           env=dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1"))
        sec = json.loads(r.stdout.strip().splitlines()[-1])["seconds"]
        scale = float(h2.sum() / h2[picks].sum())
        out["cpu_baseline"] = {"value": sec * scale, "unit": "s", "cores": 1, "kind": "oracle",
                               "sample": f"32 of the 512 instances (every 16th by size), {sec:.1f} s, scaled by "
                                         f"sum(h^2) over all / over the sample = {scale:.1f}"}
    return out


# ---------------------------------------------------------------- the reference arm (the oracle)
def run_reference(args, rank, world):
    if rank != 0:
        return
    w = workload(args.workload)
    g = os.path.join(GOLDEN, f"{args.workload}.json")
    rec = json.load(open(g)).get("tol_1e-8", {}) if os.path.exists(g) else {}
    full = rec.get("n_matvec", 707) + rec.get("n_resid_matvec", 0)
    restarts = 3
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; warm-up steps are skipped
    times = []
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    for _ in range(args.steps):
        cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", args.workload,
               "--sample-restarts", str(restarts)]
        r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        times.append(d["seconds"] * full / d["products"])
    value = statistics.mean(times)
    line = {"impl": "reference", "metric": metric_name(w), "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args.workload, w),
            "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": f"each step: first {restarts} outer iterations, scaled to the oracle's "
                                       f"{full} products A v of the whole solve"},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def metric_name(w):
    return (f"time to {w['nev']} eigenpairs at resid<=1e-8 (J-TRLan, plain FP64)")


def config_of(name, w):
    return {"workload": name, "n": 6 * inputs.lattice_volume(w["dims"]), "lattice": list(w["dims"]),
            "nev": w["nev"], "m": w["m"], "mwin": w["mwin"], "tol": TOL, "m0": w["m0"], "kappa": w["kappa"],
            "precision": "fp64", "inputs": "seeded Haar SU(3) U, complex Gaussian W",
            "l2": "flushed before every timed step (512 MB write, then a 512 MB read of another buffer)"}


# ---------------------------------------------------------------- our arm
def run_gb300(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2001_07428_gb300 import binding as B

    B.load()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    peaks = B.jtrlan_measure_peaks(torch.cuda.current_stream(dev).cuda_stream)
    fp64_peak, fp64_src = fp64_peak_tflops(peaks)
    w = workload(args.workload)
    dims = w["dims"]
    U, W = inputs.stencil_links(dims, w["seed"])
    n = 6 * inputs.lattice_volume(dims)
    Ud = torch.from_numpy(U).to(dev)
    Wd = torch.from_numpy(W).to(dev)
    stream = torch.cuda.current_stream(dev)
    op = B.stencil_operator(dims, w["m0"], w["kappa"], Ud.data_ptr(), Wd.data_ptr())
    prm = B.params(w["nev"], w["m"], w["mwin"], TOL)
    ctx = B.jtrlan_create(op, prm, stream.cuda_stream)
    flush = L2Flush(torch, dev)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        st = B.jtrlan_solve(ctx)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches = 0
    stats = []
    clocks = Clocks(local_rank)
    barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush()
        ev0[i].record(stream)
        st = B.jtrlan_solve(ctx)
        ev1[i].record(stream)
        launches += st["n_launches"]
        stats.append(st)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    times = [a.elapsed_time(b) / 1e3 for a, b in zip(ev0, ev1)]
    t_mean = max_over_ranks(statistics.mean(times), world, dev)

    # ---- the chosen (mixed-precision) form on the same workload: time and agreement with FP64
    ev64 = np.zeros(w["nev"])
    B.jtrlan_pairs(ctx, 0, ev64.ctypes.data_as(__import__("ctypes").c_void_p), None, None)
    forms = {"mixed_reorth": (B.JTRLAN_MIXED_REORTH, "FP64 vectors and matvec; reorthogonalisation in compensated "
                                                     "FP32 (double-float) on a (hi, lo) basis; FP64 alpha/beta, Ritz "
                                                     "solve, residuals"),
             "mixed": (B.JTRLAN_MIXED, "FP32 phase (matvec, GS, rotation in FP32) to max(tol, 1e-5 max|t|), then "
                                       "mixed_reorth from the summed FP32 Ritz vectors")}
    mixed = {}
    for name, (prec, desc) in forms.items():
        ctxm = B.jtrlan_create(op, B.params(w["nev"], w["m"], w["mwin"], TOL, precision=prec), stream.cuda_stream)
        for _ in range(args.warmup):
            stm = B.jtrlan_solve(ctxm)
        tm = []
        for i in range(args.steps):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stm = B.jtrlan_solve(ctxm)
            e1.record(stream)
            torch.cuda.synchronize()
            tm.append(e0.elapsed_time(e1) / 1e3)
        evm = np.zeros(w["nev"])
        B.jtrlan_pairs(ctxm, 0, evm.ctypes.data_as(__import__("ctypes").c_void_p), None, None)
        B.jtrlan_destroy(ctxm)
        t_m = statistics.mean(tm)
        mixed[name] = {"value": t_m, "unit": "s", "speedup_vs_fp64": round(t_mean / t_m, 3),
                       "n_matvec_fp32": stm["n_matvec_fp32"], "n_matvec_fp64": stm["n_matvec"] - stm["n_matvec_fp32"],
                       "n_restarts": stm["n_restarts"],
                       "max_rel_eig_diff_vs_fp64": float(np.max(np.abs(evm - ev64) / np.abs(ev64))), "form": desc}
    mixed["chosen"] = min((k for k in forms), key=lambda k: mixed[k]["value"])
    invert = invert_compare(B, torch, stream, flush, op, w, t_mean, ev64)

    # ---- one profiled solve per form: per-kernel device time
    def profiled_ctx(ctxp):
        """one solve of a context created with profile=1: per-kernel-class device time, launches,
        share and (where the work per unit is defined) achieved TFLOP/s and GB/s"""
        flush()
        torch.cuda.synchronize()
        B.jtrlan_solve(ctxp)
        prof = B.jtrlan_get_profile(ctxp)
        tot_ms = sum(v["ms"] for v in prof.values())
        out = {}
        for k, v in prof.items():
            if v["launches"] == 0:
                continue
            e = {"ms": round(v["ms"], 3), "launches": v["launches"], "share": round(v["ms"] / tot_ms, 4)}
            if k in FLOP_PER_UNIT and v["ms"] > 0:
                e["tflops"] = round(v["work"] * FLOP_PER_UNIT[k] / (v["ms"] * 1e-3) / 1e12, 4)
            if k in BYTES_PER_UNIT and v["ms"] > 0:
                e["gbs"] = round(v["work"] * BYTES_PER_UNIT[k] / (v["ms"] * 1e-3) / 1e9, 1)
            out[k] = e
        return out

    def profiled(precision):
        ctxp = B.jtrlan_create(op, B.params(w["nev"], w["m"], w["mwin"], TOL, precision=precision, profile=1),
                               stream.cuda_stream)
        out = profiled_ctx(ctxp)
        B.jtrlan_destroy(ctxp)
        return out

    kernels = profiled(B.JTRLAN_FP64)
    mixed["kernels_" + mixed["chosen"]] = profiled(forms[mixed["chosen"]][0])
    if not args.no_mixed_16:
        mixed["stencil_16x16x16x16"] = mixed_at_16(B, torch, stream, flush, profiled_ctx)
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    hbm_peak, hbm_src = measured_peaks()
    if "tflops" in kernels[dom]:
        ach = kernels[dom]["tflops"]
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": round(fp64_peak, 3),
                "unit": "TFLOP/s", "frac": round(ach / fp64_peak, 4),
                "traffic": ncu_traffic(dom, args.workload),
                "peak_source": fp64_src}
    else:
        roof = {"kernel": dom, "bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None}
    mvk = kernels.get("matvec", {})
    stencil = {"gbs": mvk.get("gbs"), "frac_of_hbm": round(mvk["gbs"] / hbm_peak, 4) if mvk.get("gbs") else None,
               "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src, "tflops": mvk.get("tflops"),
               "frac_of_fp64": round(mvk["tflops"] / fp64_peak, 4) if mvk.get("tflops") else None,
               "note": "8^4 in c128 is L2-resident (5.5 MB) and FP64-ALU-bound; GB/s counts 84 words/site"}

    # ---- end to end through the C ABI from pinned host buffers
    Uh = torch.from_numpy(U).pin_memory()
    Wh = torch.from_numpy(W).pin_memory()
    Xh = torch.empty((w["nev"], n), dtype=torch.complex128).pin_memory()
    evh = np.zeros(w["nev"])
    resh = np.zeros(w["nev"])
    op_h = B.stencil_operator(dims, w["m0"], w["kappa"], Uh.data_ptr(), Wh.data_ptr())
    import ctypes
    e2e = []
    torch.cuda.synchronize()
    for i in range(max(1, args.steps)):
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = B.jtrlan_create(op_h, prm, stream.cuda_stream)
        B.jtrlan_solve(c2)
        B.jtrlan_pairs(c2, 0, evh.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(Xh.data_ptr()),
                       resh.ctypes.data_as(ctypes.c_void_p))
        B.jtrlan_destroy(c2)
        e2e.append(time.perf_counter() - t0)
    e2e_mean = max_over_ranks(statistics.mean(e2e), world, dev)
    h2d = Uh.numel() * 16 + Wh.numel() * 16
    d2h = Xh.numel() * 16 + 2 * w["nev"] * 8
    B.jtrlan_destroy(ctx)

    if rank != 0:
        return
    line = {"metric": metric_name(w), "value": t_mean, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_mean * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_of(args.workload, w),
            "solve_stats": {k: stats[-1][k] for k in ("n_matvec", "n_resid_matvec", "n_gs_passes", "n_restarts",
                                                       "icnv", "n_ritz_fallbacks")},
            "step_ms": [round(x * 1e3, 3) for x in times],
            "gpu_launches": int(launches), "clocks": clk, "roofline": roof, "mixed": mixed, "stencil_matvec": stencil,
            "kernels": kernels,
            "e2e": {"value": e2e_mean, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}}
    line["invert_mode"] = invert
    line["stencil_fp32"] = {k: stencil_apply_roofline(v) for k, v in STENCIL_LATTICES.items()}
    line["rotate_tc"] = {k: rotate_roofline(v) for k, v in ROTATE_SHAPES.items()}
    if not args.no_learned:
        line["learned_filter"] = learned_compare(B, torch, "16x16x16x16", with_fp64=False)
    if not args.no_batched:
        line["batched_dense"] = batched_dense(B, torch, stream, args.steps, args.warmup, peaks=peaks,
                                              cpu=world == 1 and not args.no_cpu_baseline)
    if world == 1 and not args.no_cpu_baseline:
        # the oracle's own product count for the whole solve (it re-verifies locked pairs every
        # restart, as Algorithm 1 is written), from the stored oracle run when there is one
        g = os.path.join(GOLDEN, f"{args.workload}.json")
        rec = json.load(open(g)).get("tol_1e-8", {}) if os.path.exists(g) else {}
        full = (rec["n_matvec"] + rec["n_resid_matvec"]) if "n_resid_matvec" in rec else \
            stats[-1]["n_matvec"] + stats[-1]["n_resid_matvec"]
        line["cpu_baseline"] = cpu_baseline(args.workload, full)
    print(json.dumps(line), flush=True)


# ================================================================ the largest workload: learned-filter form
HEADLINE = "stencil_24x24x24x48"
FP32_LANES = 152 * 128          # SMs x FP32 lanes per SM (4 partitions x 32)


def fp32_peak_ops(peaks=None):
    """FP32 issue peak in operations/s (one FMA, add or multiply per lane per clock): measured by the
    library's FMA loop when `peaks` holds it (FMA counted as one operation), else 152 SMs x 128 lanes
    at the maximum SM clock.  Returns (ops/s, source)."""
    if peaks and peaks.get("fp32_fma_tflops"):
        return peaks["fp32_fma_tflops"] / 2 * 1e12, "measured: FP32 FMA loop (jtrlan_measure_peaks), one op per FMA"
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        mhz = float(json.load(open(p)).get("sm_max_mhz", mhz))
    return FP32_LANES * mhz * 1e6, "derived: 152 SMs x 128 lanes x max SM clock"


# Algorithmic work per unit of each kernel class of the learned-filter solve (units from the library's
# jtrlan_profile work counters), with the roof that bounds it.
#   matvec: the compensated stencil product fused with one Chebyshev step (per lattice site): 1152 real
#     products (288 complex multiply-adds of 3x3 complex64 links by neighbour colour vectors, both
#     halves) carried as biased block sums, 5 FP32 ops each (FMA into the biased sum, the exact amount
#     added, the FMA's rounding error, two into the error sum) = 5760; the bounds of the 12 blocks per
#     site (one per direction and colour row: 42 ops each) = 504; the rebias of 8 running sums per block
#     (5 ops each) = 480; the biases (3 FP32 ops each, 2 per block) = 72; the start and the removal of the
#     bias = 33; the float-float recurrence epilogue (about 150 ops per (site, colour)) = 450:
#     7,299 FP32 ops per site, against the FP32 issue rate ("alu").
#   gs_first, gs_dot, gs_update: per (row pair x basis column) the two (hi, lo) complex entries of V
#     read from HBM, 32 B ("hbm").
#   rotate: per real multiply-add of V_m Z, 2 flop FP64-equivalent; issued on the tensor cores as
#     28 BF16 digit-pair products (56 flop), against the measured BF16 peak ("tensor").
LEARNED_UNIT_WORK = {
    "matvec": ("alu", 1152 * 5 + 504 + 480 + 72 + 33 + 450, "FP32 op"),
    "gs_first": ("hbm", 32.0, "B"), "gs_dot": ("hbm", 32.0, "B"), "gs_update": ("hbm", 32.0, "B"),
    "rotate": ("tensor", 28.0, "flop"),     # x the FP64-equivalent flop count 2 n m kk of the work counter
}


def learned_roofline(kernels, workload_name, peaks=None):
    """The roofline object for the kernel class with the largest device time of a profiled step."""
    hbm, hsrc = measured_peaks()
    dom = max((k for k in kernels if k in LEARNED_UNIT_WORK), key=lambda k: kernels[k]["ms"])
    e = kernels[dom]
    bound, per_unit, unit = LEARNED_UNIT_WORK[dom]
    sec = e["ms"] * 1e-3
    out = {"kernel": dom, "bound": bound, "launches": e["launches"], "avg_launch_us": round(e["ms"] * 1e3 / e["launches"], 2)}
    if bound == "hbm":
        ach = e["work"] * per_unit / sec / 1e9
        out.update(achieved=round(ach, 1), peak=hbm, unit="GB/s", frac=round(ach / hbm, 4),
                   peak_source=f"{hsrc} (MEASURED_PEAKS.json hbm_gbs)")
    elif bound == "alu":
        peak, psrc = fp32_peak_ops(peaks)
        peak /= 1e12
        ach = e["work"] * per_unit / sec / 1e12
        out.update(achieved=round(ach, 2), peak=round(peak, 2), unit="Tops/s", frac=round(ach / peak, 4),
                   peak_source=psrc, work="FP32 ops of the compensated arithmetic as written, per lattice site")
    else:
        peak, src = bf16_peak()
        ach = e["work"] * per_unit / sec / 1e12
        out.update(achieved=round(ach, 1), peak=peak, unit="TFLOP/s", frac=round(ach / peak, 4), peak_source=src)
    out["traffic"] = ncu_traffic(dom, workload_name)
    return out


def profile_table(prof):
    tot = sum(v["ms"] for v in prof.values()) or 1.0
    return {k: {"ms": round(v["ms"], 3), "launches": v["launches"], "share": round(v["ms"] / tot, 4),
                "work": v["work"]} for k, v in prof.items() if v["launches"]}


def oracle_primitives(name, steps=6, rot_rows_div=64):
    """Times the oracle's pieces on the full-size workload (run as a subprocess): one stencil product,
    Algorithm 2 one step at a time for j = 0 .. steps-1 (each step's product timed apart, the rest is
    its Gram-Schmidt against j + 1 columns of V and W), and the restart rotation V_m Z on 1/rot_rows_div
    of the rows.  Returns seconds per product, per Gram-Schmidt column (one pass), per full rotation."""
    from oracle import jsym
    from oracle import trlan_jsym as tj
    w = workload(name)
    dims = w["dims"]
    U, W = inputs.stencil_links(dims, w["seed"])
    if w.get("links") == "c64":
        U, W = U.astype(np.complex64).astype(np.complex128), W.astype(np.complex64).astype(np.complex128)
    n = 6 * inputs.lattice_volume(dims)
    mv_t = []

    def mv(x):
        t0 = time.perf_counter()
        y = jsym.stencil_matvec(U, W, dims, w["m0"], w["kappa"], x)
        mv_t.append(time.perf_counter() - t0)
        return y

    V = np.zeros((n, steps + 1), dtype=np.complex128)
    T = np.zeros((steps + 1, steps + 1))
    V[:, 0] = 1.0 / np.sqrt(n)
    per_col = []
    t_all = time.perf_counter()
    for j in range(steps):
        st = dict(n_matvec=0, n_gs_passes=0)
        t0 = time.perf_counter()
        tj.lanczos_jsym(mv, V, T, j, j + 1, stats=st)
        gs = time.perf_counter() - t0 - mv_t[-1]
        per_col.append(gs / (st["n_gs_passes"] * (j + 1)))
    m, kk = w["m"], w["m"]
    rows = n // rot_rows_div
    Z = np.linalg.qr(np.random.default_rng(0).standard_normal((m, m)))[0]
    Vs = (np.random.default_rng(1).standard_normal((rows, m)) + 0j)
    t0 = time.perf_counter()
    _ = Vs @ Z
    t_rot = (time.perf_counter() - t0) * rot_rows_div
    sampled = time.perf_counter() - t_all
    return {"t_matvec": float(np.median(mv_t)), "t_gs_col": float(np.median(per_col)), "t_rotate": t_rot,
            "sample_seconds": sampled, "steps": steps, "n": n}


def cpu_projection(name, counts, threads):
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-primitives", name]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        return {"value": None, "error": r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    prods = counts["n_matvec"] + counts["n_resid_matvec"]
    proj = prods * d["t_matvec"] + counts["gs_column_passes"] * d["t_gs_col"] + counts["n_restarts"] * d["t_rotate"]
    return {"value": proj, "unit": "s", "cores": threads, "kind": "oracle",
            "sample": (f"oracle pieces timed on the full-size workload ({d['sample_seconds']:.1f} s): one stencil "
                       f"product {d['t_matvec']:.2f} s, Algorithm 2 for {d['steps']} single steps "
                       f"({d['t_gs_col'] * 1e3:.1f} ms per Gram-Schmidt column and pass), the rotation V_m Z on "
                       f"1/64 of the rows ({d['t_rotate']:.1f} s scaled); projected with the plain FP64 GPU "
                       f"solve's counts: {prods} products, {counts['gs_column_passes']:.0f} column passes, "
                       f"{counts['n_restarts']} rotations"),
            "measured": d, "counts": counts}


def run_headline(args, rank, world, local_rank):
    import ctypes

    import torch
    import torch.distributed as dist

    from paper_2001_07428_gb300 import binding as B
    from paper_2001_07428_gb300 import learned_filter as LF

    t_begin = time.perf_counter()
    B.load()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    peaks = B.jtrlan_measure_peaks(torch.cuda.current_stream(dev).cuda_stream)
    name = args.workload
    w = workload(name)
    dims, nev, m, mwin = w["dims"], w["nev"], w["m"], w["mwin"]
    vol = inputs.lattice_volume(dims)
    n = 6 * vol
    U, W = inputs.stencil_links(dims, w["seed"])
    U, W = U.astype(np.complex64), W.astype(np.complex64)
    Ud, Wd = torch.from_numpy(U).to(dev), torch.from_numpy(W).to(dev)
    stream = torch.cuda.current_stream(dev)
    op = B.stencil_operator(dims, w["m0"], w["kappa"], Ud.data_ptr(), Wd.data_ptr(), dtype=B.JTRLAN_C64)
    net = LF.FilterNet.load(device=dev)
    prm = B.params(nev, m, mwin, TOL, precision=B.JTRLAN_MIXED_REORTH)
    ctx = B.jtrlan_create(op, prm, stream.cuda_stream)
    flush = L2Flush(torch, dev)

    def step(c):
        """bounds on the context, inference, the filter set on the context, the solve"""
        g, win, _ = LF.filter_on_context(net, c, w["m0"], w["kappa"], nev, vol)
        nb = sum(v["launches"] for v in B.jtrlan_get_profile(c).values()) + 3   # bounds + 3 MLP layers
        st = B.jtrlan_solve(c)
        return st, nb + st["n_launches"], g, win

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step(ctx)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches, stats = 0, []
    clocks = Clocks(local_rank)
    barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush()
        ev0[i].record(stream)
        st, nl, g, win = step(ctx)
        ev1[i].record(stream)
        launches += nl
        stats.append(st)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    times = [a.elapsed_time(b) / 1e3 for a, b in zip(ev0, ev1)]
    t_mean = max_over_ranks(statistics.mean(times), world, dev)
    ev_l, res_l = np.zeros(nev), np.zeros(nev)
    B.jtrlan_pairs(ctx, 0, ev_l.ctypes.data_as(ctypes.c_void_p), None, res_l.ctypes.data_as(ctypes.c_void_p))
    t_timed_end = time.perf_counter()

    # ---- one profiled step: per-kernel-class device time, and the roofline of the dominant class
    ctxp = B.jtrlan_create(op, B.params(nev, m, mwin, TOL, precision=B.JTRLAN_MIXED_REORTH, profile=1),
                           stream.cuda_stream)
    flush()
    step(ctxp)
    kernels = profile_table(B.jtrlan_get_profile(ctxp))
    B.jtrlan_destroy(ctxp)
    roof = learned_roofline(kernels, name, peaks)

    # ---- the FP32 stencil matvec of this lattice against the measured HBM peak
    stencil = stencil_apply_roofline(dims)

    # ---- end to end through the C ABI from pinned host buffers
    Uh, Wh = torch.from_numpy(U).pin_memory(), torch.from_numpy(W).pin_memory()
    Xh = torch.empty((nev, n), dtype=torch.complex128).pin_memory()
    evh, resh = np.zeros(nev), np.zeros(nev)
    op_h = B.stencil_operator(dims, w["m0"], w["kappa"], Uh.data_ptr(), Wh.data_ptr(), dtype=B.JTRLAN_C64)
    e2e = []
    for _ in range(args.e2e_steps):
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = B.jtrlan_create(op_h, prm, stream.cuda_stream)
        step(c2)
        B.jtrlan_pairs(c2, 0, evh.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(Xh.data_ptr()),
                       resh.ctypes.data_as(ctypes.c_void_p))
        B.jtrlan_destroy(c2)
        e2e.append(time.perf_counter() - t0)
    e2e_mean = max_over_ranks(statistics.mean(e2e), world, dev)
    h2d = Uh.numel() * 8 + Wh.numel() * 8
    d2h = Xh.numel() * 16 + 2 * nev * 8
    del Xh
    B.jtrlan_destroy(ctx)

    # ---- plain FP64 J-TRLan on the same workload and GPU (same complex64 links, FP64 arithmetic)
    fp64 = None
    if not args.no_fp64:
        c64 = B.jtrlan_create(op, B.params(nev, m, mwin, TOL, precision=B.JTRLAN_FP64), stream.cuda_stream)
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st64 = B.jtrlan_solve(c64)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        ev64, res64 = np.zeros(nev), np.zeros(nev)
        B.jtrlan_pairs(c64, 0, ev64.ctypes.data_as(ctypes.c_void_p), None, res64.ctypes.data_as(ctypes.c_void_p))
        prof64 = B.jtrlan_get_profile(c64)
        B.jtrlan_destroy(c64)
        h = n // 2
        colpasses = sum(prof64[k]["work"] for k in ("gs_first", "gs_dot", "gs_update") if k in prof64) / h / 2
        rel = np.abs(ev_l - ev64) / np.abs(ev64)
        fp64 = {"value": t64, "unit": "s", "n_matvec": st64["n_matvec"], "n_resid_matvec": st64["n_resid_matvec"],
                "n_restarts": st64["n_restarts"], "n_gs_passes": st64["n_gs_passes"],
                "max_residual": float(res64.max()), "speedup_of_learned_form": round(t64 / t_mean, 3),
                "rel_eig_diff_learned_vs_fp64": [float("%.3g" % v) for v in rel],
                "max_rel_eig_diff": float(rel.max()), "eigenvalues_fp64": [float(v) for v in ev64],
                "gs_column_passes": colpasses}
    t_end_gpu = time.perf_counter()

    if rank != 0:
        return
    last = stats[-1]
    line = {"metric": f"time to {nev} eigenpairs at resid<=1e-8 (learned-filter mixed-precision J-TRLan)",
            "value": t_mean, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_mean * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 vectors + compensated f32 (double-float) products and Gram-Schmidt + bf16-digit "
                     "tensor MMA rotation; f32 network",
            "data": "synthetic",
            "config": {"workload": name, "n": n, "lattice": list(dims), "nev": nev, "m": m, "mwin": mwin, "tol": TOL,
                       "m0": w["m0"], "kappa": w["kappa"], "links": "complex64 (seeded Haar SU(3) U, complex "
                       "Gaussian W, rounded)", "form": "learned filter (degree %d) + JTRLAN_MIXED_REORTH" % (len(g) - 1),
                       "l2": "flushed before every timed step (512 MB write, then a 512 MB read of another buffer); "
                             "the basis (12.9 GB) exceeds L2 in any case"},
            "solve_stats": {k: last[k] for k in ("n_matvec", "n_resid_matvec", "n_gs_passes", "n_restarts", "icnv",
                                                 "n_ritz_fallbacks")},
            "step_s": [round(x, 4) for x in times], "max_residual": float(res_l.max()),
            "filter": {"degree": len(g) - 1, "window": list(win), "cut_tau": float(np.cos(np.pi * (1 - g[0])))},
            "gpu_launches": int(launches), "clocks": clk, "roofline": roof, "kernels": kernels,
            "measured_peaks": {k: round(v, 3) for k, v in peaks.items()},
            "stencil_fp32": stencil, "vs_plain_fp64": fp64,
            "e2e": {"value": e2e_mean, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "steps": args.e2e_steps},
            "wall_s": {"to_end_of_timed_steps": round(t_timed_end - t_begin, 1),
                       "gpu_part": round(t_end_gpu - t_begin, 1)}}
    if world == 1 and not args.no_cpu_baseline and fp64 is not None:
        counts = {"n_matvec": fp64["n_matvec"], "n_resid_matvec": fp64["n_resid_matvec"],
                  "n_restarts": fp64["n_restarts"], "gs_column_passes": fp64["gs_column_passes"]}
        one = cpu_projection(name, counts, 1)
        ncpu = os.cpu_count() or 1
        allc = cpu_projection(name, counts, ncpu)
        one["nproc"] = ncpu
        one["all_cores"] = {k: allc.get(k) for k in ("value", "cores", "measured")}
        one["all_cores"]["note"] = ("same oracle, BLAS allowed all host threads (numpy's element-wise "
                                    "operations stay on one thread)")
        line["cpu_baseline"] = one
    line["wall_s"]["total"] = round(time.perf_counter() - t_begin, 1)
    print(json.dumps(line), flush=True)


def run_reference_headline(args, rank, world):
    """The oracle as the reference arm on the full-size workload: every step (warm-up steps included)
    is one Lanczos step of Algorithm 2 -- the stencil product and the J-reorthogonalisation against all
    columns so far -- continuing the same Krylov sequence, timed as measured (not projected)."""
    if rank != 0:
        return
    from oracle import jsym
    from oracle import trlan_jsym as tj
    name = args.workload
    w = workload(name)
    dims = w["dims"]
    U, W = inputs.stencil_links(dims, w["seed"])
    U, W = U.astype(np.complex64).astype(np.complex128), W.astype(np.complex64).astype(np.complex128)
    n = 6 * inputs.lattice_volume(dims)
    mv = lambda x: jsym.stencil_matvec(U, W, dims, w["m0"], w["kappa"], x)
    total = args.warmup + args.steps
    V = np.zeros((n, total + 1), dtype=np.complex128)
    T = np.zeros((total + 1, total + 1))
    V[:, 0] = 1.0 / np.sqrt(n)
    times = []
    for j in range(total):
        t0 = time.perf_counter()
        tj.lanczos_jsym(mv, V, T, j, j + 1)
        if j >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = statistics.mean(times)
    threads = os.environ.get("OPENBLAS_NUM_THREADS", "default")
    line = {"impl": "reference",
            "metric": f"time to {w['nev']} eigenpairs at resid<=1e-8 (learned-filter mixed-precision J-TRLan)",
            "value": value, "unit": "s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "n": n, "lattice": list(dims), "nev": w["nev"], "m": w["m"],
                       "mwin": w["mwin"], "tol": TOL, "links": "complex64"},
            "value_is": ("measured seconds per sampled step: one Lanczos step (Algorithm 2) of the CPU FP64 oracle "
                         "at full size, steps %d..%d of one Krylov sequence from v1 = 1/||1|| (Gram-Schmidt "
                         "against %d..%d columns of V and W); not a time to solution" %
                         (args.warmup, total - 1, args.warmup + 1, total)),
            "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle", "nproc": os.cpu_count(),
                             "blas_threads": threads,
                             "sample": "one oracle Lanczos step at full size per step (see value_is)"},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "step_s": [round(t, 3) for t in times]}
    print(json.dumps(line), flush=True)



def one_step(args):
    """One step of the learned-filter form on a workload (for profilers): context, bounds, inference,
    set_filter, solve; prints the step's time and counters.  --gs-split forces the separate-launch
    Gram-Schmidt; --max-restarts bounds the solve (a bounded solve that stops early still exits 0)."""
    import ctypes

    import torch

    from paper_2001_07428_gb300 import binding as B
    from paper_2001_07428_gb300 import learned_filter as LF
    B.load()
    dev = torch.device("cuda", 0)
    w = workload(args.one_step)
    dims, nev, m, mwin = w["dims"], w["nev"], w["m"], w["mwin"]
    if args.nev:        # a smaller basis keeps a profiler's device memory small; kernels per launch unchanged
        nev, m = args.nev, args.m or 2 * args.nev
        mwin = min(2 * nev, m // 2)
    vol = inputs.lattice_volume(dims)
    U, W = inputs.stencil_links(dims, w["seed"])
    U, W = U.astype(np.complex64), W.astype(np.complex64)
    Ud, Wd = torch.from_numpy(U).to(dev), torch.from_numpy(W).to(dev)
    stream = torch.cuda.current_stream(dev)
    op = B.stencil_operator(dims, w["m0"], w["kappa"], Ud.data_ptr(), Wd.data_ptr(), dtype=B.JTRLAN_C64)
    net = LF.FilterNet.load(device=dev)
    ctx = B.jtrlan_create(op, B.params(nev, m, mwin, TOL, precision=B.JTRLAN_MIXED_REORTH,
                                       max_restarts=args.max_restarts, gs_split=int(args.gs_split)),
                          stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g, win, _ = LF.filter_on_context(net, ctx, w["m0"], w["kappa"], nev, vol)
    status = "ok"
    try:
        st = B.jtrlan_solve(ctx)
    except B.JTRLanError as e:
        if e.status != B.JTRLAN_ENOCONV:
            raise
        status, st = "stopped at max_restarts", {}
    torch.cuda.synchronize()
    out = {"workload": args.one_step, "nev": nev, "m": m, "seconds": time.perf_counter() - t0, "status": status,
           "degree": len(g) - 1,
           "gs_split": bool(args.gs_split), "max_restarts": args.max_restarts,
           **{k: st.get(k) for k in ("n_matvec", "n_restarts", "n_gs_passes", "n_launches")}}
    B.jtrlan_destroy(ctx)
    print(json.dumps(out), flush=True)



def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=HEADLINE)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 solve of the largest workload")
    ap.add_argument("--e2e-steps", type=int, default=1, help="end-to-end steps through the C ABI (largest workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed-16", action="store_true", help="skip the 16^4 FP64 vs mixed comparison")
    ap.add_argument("--stencil-only", default=None, choices=sorted(STENCIL_LATTICES),
                    help="only time the FP32 stencil matvec on this lattice (for profiling)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched dense instances")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-filter comparison at 16^4")
    ap.add_argument("--learned-only", default=None, choices=sorted(LEARNED_LATTICES),
                    help="only compare the learned-filter form with the unfiltered solver on this lattice")
    ap.add_argument("--with-fp64", action="store_true", help="with --learned-only: also time plain FP64")
    ap.add_argument("--rotate-only", default=None, choices=sorted(ROTATE_SHAPES),
                    help="only time the restart rotation of the (hi, lo) basis at this lattice's shape")
    ap.add_argument("--batched-only", action="store_true", help="only time the batched dense instances")
    ap.add_argument("--batch-count", type=int, default=None, help="with --batched-only: the first N instances")
    ap.add_argument("--batch-shape", default=None, help="with --batched-only: THREADS,CTAS_PER_SM instead of tuning")
    ap.add_argument("--batch-forms", default="fp64,mixed_reorth", help="with --batched-only: forms to time")
    ap.add_argument("--case-a", action="store_true", help="only run the Case A sweep (TRLAN-JSYM vs plain TRLAN)")
    ap.add_argument("--batched-oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--sample-restarts", type=int, default=4, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-primitives", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--one-step", default=None, help="one learned-filter step on this workload (for profilers)")
    ap.add_argument("--gs-split", action="store_true", help="with --one-step: separate-launch Gram-Schmidt")
    ap.add_argument("--max-restarts", type=int, default=0, help="with --one-step: bound on outer iterations")
    ap.add_argument("--nev", type=int, default=0, help="with --one-step: nev instead of the workload's")
    ap.add_argument("--m", type=int, default=0, help="with --one-step and --nev: m (default 2 nev)")
    args = ap.parse_args()
    if args.batched_oracle_sample:
        print(json.dumps({"seconds": batched_oracle_sample([int(i) for i in args.batched_oracle_sample.split(",")])}))
        return
    if args.one_step:
        one_step(args)
        return
    if args.oracle_primitives:
        print(json.dumps(oracle_primitives(args.oracle_primitives)))
        return
    if args.oracle_sample:
        sec, done = oracle_sample(args.oracle_sample, args.sample_restarts)
        print(json.dumps({"seconds": sec, "products": done}))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if args.workload == HEADLINE:
            run_reference_headline(args, rank, world)
        else:
            run_reference(args, rank, world)
        return
    if args.rotate_only:
        print(json.dumps(rotate_roofline(ROTATE_SHAPES[args.rotate_only])), flush=True)
        return
    if args.stencil_only:
        print(json.dumps(stencil_apply_roofline(STENCIL_LATTICES[args.stencil_only])), flush=True)
        return
    if args.case_a:
        import torch
        from paper_2001_07428_gb300 import binding as B
        B.load()
        print(json.dumps(case_a_sweep(B, torch)), flush=True)
        return
    if args.learned_only:
        import torch
        from paper_2001_07428_gb300 import binding as B
        B.load()
        print(json.dumps(learned_compare(B, torch, args.learned_only, with_fp64=args.with_fp64)), flush=True)
        return
    if args.batched_only:
        import torch
        from paper_2001_07428_gb300 import binding as B
        B.load()
        shape = tuple(int(v) for v in args.batch_shape.split(",")) if args.batch_shape else None
        peaks = B.jtrlan_measure_peaks(torch.cuda.current_stream().cuda_stream)
        print(json.dumps(batched_dense(B, torch, torch.cuda.current_stream(), args.steps, args.warmup, peaks=peaks,
                                       cpu=not args.no_cpu_baseline, count=args.batch_count, shape=shape,
                                       forms=tuple(args.batch_forms.split(",")))), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        if args.workload == HEADLINE:
            run_headline(args, rank, world, local_rank)
        else:
            run_gb300(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
