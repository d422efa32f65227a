"""Thin ctypes binding over libjtrlan.so (C ABI in include/jtrlan.h).

Only argument marshalling lives here: every step of the solver runs in the library's CUDA
kernels.  Buffers are passed as raw pointers -- ``torch.Tensor.data_ptr()`` for device (or pinned
host) tensors, ``numpy.ndarray.ctypes.data`` for host arrays.  There is no CPU fallback: if the
library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libjtrlan.so")

JTRLAN_OK, JTRLAN_EINVAL, JTRLAN_ENOMEM, JTRLAN_ECUDA, JTRLAN_ENOTJSYM = 0, 1, 2, 3, 4
JTRLAN_EBREAKDOWN, JTRLAN_ENOCONV, JTRLAN_ETIMEOUT, JTRLAN_ESTATE = 5, 6, 7, 8
JTRLAN_DENSE, JTRLAN_STENCIL4D = 0, 1
JTRLAN_C128, JTRLAN_C64 = 0, 1
JTRLAN_SMALLEST, JTRLAN_LARGEST = 0, 1
JTRLAN_FP64, JTRLAN_MIXED, JTRLAN_MIXED_REORTH = 0, 1, 2

EXPORTED = ["jtrlan_create", "jtrlan_apply", "jtrlan_solve", "jtrlan_pairs", "jtrlan_get_profile",
            "jtrlan_residual_norms_noalloc", "jtrlan_destroy", "jtrlan_status_string", "jtrlan_last_error",
            "jtrlan_batch_create", "jtrlan_batch_set_shape", "jtrlan_batch_tune", "jtrlan_batch_solve",
            "jtrlan_batch_results", "jtrlan_batch_vectors", "jtrlan_batch_destroy", "jtrlan_apply_filter", "jtrlan_bounds",
            "jtrlan_damped_step", "jtrlan_mlp_param_count", "jtrlan_mlp_create", "jtrlan_mlp_get_params",
            "jtrlan_mlp_set_params", "jtrlan_mlp_forward", "jtrlan_mlp_gradient", "jtrlan_mlp_train",
            "jtrlan_mlp_destroy", "jtrlan_rotate_df", "jtrlan_set_filter", "jtrlan_measure_peaks",
            "jtrlan_batch_set_tiles", "jtrlan_batch_get_tiles"]
NOALLOC_MAX_PARTIALS = 262144   # JTRLAN_NOALLOC_MAX_PARTIALS
NOALLOC_MAX_COLS = 1024         # JTRLAN_NOALLOC_MAX_COLS


class jtrlan_operator(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dtype", ctypes.c_int), ("n", ctypes.c_int64),
                ("dims", ctypes.c_int * 4), ("m0", ctypes.c_double), ("kappa", ctypes.c_double),
                ("a11", ctypes.c_void_p), ("a12", ctypes.c_void_p), ("U", ctypes.c_void_p),
                ("W", ctypes.c_void_p)]


class jtrlan_params(ctypes.Structure):
    _fields_ = [("nev", ctypes.c_int), ("m", ctypes.c_int), ("mwin", ctypes.c_int),
                ("tol", ctypes.c_double), ("which", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_restarts", ctypes.c_int), ("gs_max_passes", ctypes.c_int),
                ("v1", ctypes.c_void_p), ("check_jsym", ctypes.c_int), ("profile", ctypes.c_int),
                ("filter_degree", ctypes.c_int), ("filter_coeffs", ctypes.c_void_p), ("filter_lo", ctypes.c_double),
                ("filter_hi", ctypes.c_double), ("filter_final_degree", ctypes.c_int),
                ("filter_final_coeffs", ctypes.c_void_p), ("plain_trlan", ctypes.c_int),
                ("rotate_simt", ctypes.c_int), ("invert", ctypes.c_int), ("cg_tol", ctypes.c_double),
                ("cg_max_iter", ctypes.c_int), ("gs_split", ctypes.c_int)]


class jtrlan_stats(ctypes.Structure):
    _fields_ = [("n_matvec", ctypes.c_int64), ("n_resid_matvec", ctypes.c_int64),
                ("n_gs_passes", ctypes.c_int64), ("n_restarts", ctypes.c_int),
                ("icnv", ctypes.c_int), ("solve_ms", ctypes.c_double), ("n_launches", ctypes.c_int64),
                ("n_ritz_fallbacks", ctypes.c_int), ("n_restarts_fp32", ctypes.c_int),
                ("n_matvec_fp32", ctypes.c_int64), ("n_matvec_inner", ctypes.c_int64),
                ("n_cg_iters", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


MAX_KERNEL_CLASSES = 16


class jtrlan_batch_stats(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("n_ok", ctypes.c_int), ("n_matvec", ctypes.c_int64),
                ("n_resid_matvec", ctypes.c_int64), ("max_restarts", ctypes.c_int), ("grid", ctypes.c_int),
                ("threads", ctypes.c_int), ("graph", ctypes.c_int), ("solve_ms", ctypes.c_double),
                ("n_ritz_fallbacks", ctypes.c_int64), ("n_gs_passes", ctypes.c_int64),
                ("phase_frac", ctypes.c_double * 5)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["phase_frac"] = dict(zip(BATCH_PHASES, self.phase_frac))
        return d


BATCH_STATS = 6   # JTRLAN_BATCH_STATS
BATCH_PHASES = ("lanczos_product", "gram_schmidt", "ritz", "rotate_shrink", "residuals")


class jtrlan_profile(ctypes.Structure):
    _fields_ = [("n_classes", ctypes.c_int), ("names", ctypes.c_char_p * MAX_KERNEL_CLASSES),
                ("ms", ctypes.c_double * MAX_KERNEL_CLASSES),
                ("launches", ctypes.c_int64 * MAX_KERNEL_CLASSES),
                ("work", ctypes.c_double * MAX_KERNEL_CLASSES)]

    def as_dict(self):
        return {self.names[i].decode(): dict(ms=self.ms[i], launches=self.launches[i], work=self.work[i])
                for i in range(self.n_classes)}


class JTRLanError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libjtrlan.so (once); raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with python -m paper_2001_07428_gb300.build")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    lib.jtrlan_create.argtypes = [P(jtrlan_operator), P(jtrlan_params), ctypes.c_void_p,
                                  P(ctypes.c_void_p)]
    lib.jtrlan_apply.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.jtrlan_solve.argtypes = [ctypes.c_void_p, P(jtrlan_stats)]
    lib.jtrlan_pairs.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p]
    lib.jtrlan_get_profile.argtypes = [ctypes.c_void_p, P(jtrlan_profile)]
    lib.jtrlan_residual_norms_noalloc.argtypes = [P(jtrlan_operator), ctypes.c_void_p, ctypes.c_int64,
                                                  ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_void_p]
    lib.jtrlan_destroy.argtypes = [ctypes.c_void_p]
    lib.jtrlan_destroy.restype = None
    lib.jtrlan_status_string.argtypes = [ctypes.c_int]
    lib.jtrlan_status_string.restype = ctypes.c_char_p
    lib.jtrlan_last_error.argtypes = []
    lib.jtrlan_last_error.restype = ctypes.c_char_p
    lib.jtrlan_batch_create.argtypes = [ctypes.c_int, P(jtrlan_operator), P(jtrlan_params), ctypes.c_void_p,
                                        P(ctypes.c_void_p)]
    lib.jtrlan_batch_set_shape.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    lib.jtrlan_batch_tune.argtypes = [ctypes.c_void_p, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_double)]
    lib.jtrlan_batch_solve.argtypes = [ctypes.c_void_p, P(jtrlan_batch_stats)]
    lib.jtrlan_batch_set_tiles.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    lib.jtrlan_batch_get_tiles.argtypes = [ctypes.c_void_p, P(ctypes.c_int), P(ctypes.c_int)]
    lib.jtrlan_batch_results.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.jtrlan_batch_vectors.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    lib.jtrlan_batch_destroy.argtypes = [ctypes.c_void_p]
    lib.jtrlan_batch_destroy.restype = None
    lib.jtrlan_apply_filter.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.jtrlan_bounds.argtypes = [ctypes.c_void_p, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double)]
    lib.jtrlan_measure_peaks.argtypes = [P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double), ctypes.c_void_p]
    lib.jtrlan_set_filter.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
    lib.jtrlan_damped_step.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.jtrlan_mlp_param_count.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.jtrlan_mlp_param_count.restype = ctypes.c_int64
    lib.jtrlan_mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p,
                                      P(ctypes.c_void_p)]
    lib.jtrlan_mlp_get_params.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.jtrlan_mlp_set_params.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.jtrlan_mlp_forward.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    lib.jtrlan_mlp_gradient.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p, P(ctypes.c_double)]
    lib.jtrlan_mlp_train.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_float, ctypes.c_void_p]
    lib.jtrlan_mlp_destroy.argtypes = [ctypes.c_void_p]
    lib.jtrlan_mlp_destroy.restype = None
    lib.jtrlan_rotate_df.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    for f in ("jtrlan_create", "jtrlan_apply", "jtrlan_solve", "jtrlan_pairs", "jtrlan_get_profile",
              "jtrlan_residual_norms_noalloc", "jtrlan_batch_create", "jtrlan_batch_set_shape",
              "jtrlan_batch_tune", "jtrlan_batch_solve", "jtrlan_batch_results", "jtrlan_batch_vectors",
              "jtrlan_apply_filter", "jtrlan_bounds", "jtrlan_damped_step", "jtrlan_mlp_create", "jtrlan_mlp_get_params",
              "jtrlan_mlp_set_params", "jtrlan_mlp_forward", "jtrlan_mlp_gradient", "jtrlan_mlp_train",
              "jtrlan_rotate_df", "jtrlan_set_filter", "jtrlan_measure_peaks", "jtrlan_batch_set_tiles",
              "jtrlan_batch_get_tiles"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int):
    if status != JTRLAN_OK:
        lib = load()
        msg = lib.jtrlan_last_error().decode() or lib.jtrlan_status_string(status).decode()
        raise JTRLanError(status, msg)


# ---------------------------------------------------------------- the C calls, same names
def jtrlan_create(op: jtrlan_operator, params: jtrlan_params, stream: int = 0) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(load().jtrlan_create(ctypes.byref(op), ctypes.byref(params), ctypes.c_void_p(stream),
                                ctypes.byref(ctx)))
    return ctx


def jtrlan_apply(ctx, x_ptr: int, y_ptr: int):
    _check(load().jtrlan_apply(ctx, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr)))


def jtrlan_solve(ctx) -> dict:
    st = jtrlan_stats()
    _check(load().jtrlan_solve(ctx, ctypes.byref(st)))
    return st.as_dict()


def jtrlan_pairs(ctx, with_partners: int, evals_ptr, evecs_ptr, res_ptr):
    _check(load().jtrlan_pairs(ctx, int(with_partners), evals_ptr, evecs_ptr, res_ptr))


def jtrlan_get_profile(ctx) -> dict:
    pr = jtrlan_profile()
    _check(load().jtrlan_get_profile(ctx, ctypes.byref(pr)))
    return pr.as_dict()


def jtrlan_residual_norms_noalloc(op: jtrlan_operator, x_ptr: int, ldx: int, ncols: int, lambda_ptr,
                                  res_ptr, stream: int = 0):
    """||A x_i - lambda_i x_i|| for the columns of a device array, without any device allocation
    (for callers that cannot allocate device memory; see include/jtrlan.h)."""
    _check(load().jtrlan_residual_norms_noalloc(ctypes.byref(op), ctypes.c_void_p(x_ptr), int(ldx), int(ncols),
                                                lambda_ptr, res_ptr, ctypes.c_void_p(stream)))


def jtrlan_destroy(ctx):
    if ctx:
        load().jtrlan_destroy(ctx)


def jtrlan_batch_create(ops, params: jtrlan_params, stream: int = 0) -> ctypes.c_void_p:
    """ops: a sequence of jtrlan_operator (dense); copied into one contiguous array for the call."""
    arr = (jtrlan_operator * len(ops))(*ops)
    b = ctypes.c_void_p()
    _check(load().jtrlan_batch_create(len(ops), arr, ctypes.byref(params), ctypes.c_void_p(stream),
                                      ctypes.byref(b)))
    return b


def jtrlan_batch_set_shape(b, threads: int, ctas_per_sm: int):
    _check(load().jtrlan_batch_set_shape(b, int(threads), int(ctas_per_sm)))


def jtrlan_batch_tune(b) -> dict:
    t, c, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(load().jtrlan_batch_tune(b, ctypes.byref(t), ctypes.byref(c), ctypes.byref(ms)))
    return dict(threads=t.value, ctas_per_sm=c.value, best_ms=ms.value, **jtrlan_batch_get_tiles(b))


def jtrlan_batch_set_tiles(b, mv_rows: int, gs_groups: int):
    _check(load().jtrlan_batch_set_tiles(b, int(mv_rows), int(gs_groups)))


def jtrlan_batch_get_tiles(b) -> dict:
    r, g = ctypes.c_int(), ctypes.c_int()
    _check(load().jtrlan_batch_get_tiles(b, ctypes.byref(r), ctypes.byref(g)))
    return dict(mv_rows=r.value, gs_groups=g.value)


def jtrlan_batch_solve(b, check: bool = True) -> dict:
    """Returns the stats; with check=False a non-converged instance does not raise (status in 'status')."""
    st = jtrlan_batch_stats()
    status = load().jtrlan_batch_solve(b, ctypes.byref(st))
    if check:
        _check(status)
    d = st.as_dict()
    d["status"] = status
    return d


def jtrlan_batch_results(b, evals_ptr, res_ptr, istats_ptr):
    _check(load().jtrlan_batch_results(b, evals_ptr, res_ptr, istats_ptr))


def jtrlan_batch_vectors(b, i: int, evecs_ptr):
    _check(load().jtrlan_batch_vectors(b, int(i), evecs_ptr))


def jtrlan_batch_destroy(b):
    if b:
        load().jtrlan_batch_destroy(b)


def jtrlan_apply_filter(ctx, x_ptr: int, y_ptr: int):
    _check(load().jtrlan_apply_filter(ctx, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr)))


def jtrlan_bounds(ctx, steps: int):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(load().jtrlan_bounds(ctx, int(steps), ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def jtrlan_measure_peaks(stream: int = 0) -> dict:
    """Measured FP64 FMA, FP64 tensor (mma.sync m8n8k4) and FP32 FMA throughput of the device, TFLOP/s."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().jtrlan_measure_peaks(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.c_void_p(stream)))
    return {"fp64_fma_tflops": a.value, "fp64_mma_tflops": b.value, "fp32_fma_tflops": c.value}


def jtrlan_set_filter(ctx, coeffs, window):
    """The certifying phase's filter of a context: Chebyshev coefficients g_0..g_d on [lo, hi]."""
    import numpy as np
    g = np.ascontiguousarray(coeffs, dtype=np.float64)
    _check(load().jtrlan_set_filter(ctx, len(g) - 1, g.ctypes.data_as(ctypes.c_void_p), float(window[0]),
                                    float(window[1])))


def jtrlan_damped_step(tau_ptr: int, count: int, degree: int, out_ptr: int, stream: int = 0):
    _check(load().jtrlan_damped_step(ctypes.c_void_p(tau_ptr), int(count), int(degree), ctypes.c_void_p(out_ptr),
                                     ctypes.c_void_p(stream)))


def jtrlan_rotate_df(V_ptr: int, n: int, m: int, Z_ptr: int, kk: int, out_ptr: int, path: int = 0, stream: int = 0):
    """out (n x kk complex128) = V Z for a (hi, lo) basis V (n x m float4) and FP64 Z (m x kk); path 0 =
    tensor cores, 1 = CUDA cores."""
    _check(load().jtrlan_rotate_df(ctypes.c_void_p(V_ptr), int(n), int(m), ctypes.c_void_p(Z_ptr), int(kk),
                                   ctypes.c_void_p(out_ptr), int(path), ctypes.c_void_p(stream)))


def jtrlan_mlp_param_count(n_in: int, width: int, n_out: int) -> int:
    return int(load().jtrlan_mlp_param_count(int(n_in), int(width), int(n_out)))


def jtrlan_mlp_create(n_in: int, width: int, n_out: int, seed: int, stream: int = 0):
    net = ctypes.c_void_p()
    _check(load().jtrlan_mlp_create(int(n_in), int(width), int(n_out), ctypes.c_uint64(seed), ctypes.c_void_p(stream),
                                    ctypes.byref(net)))
    return net


def jtrlan_mlp_get_params(net, theta_ptr):
    _check(load().jtrlan_mlp_get_params(net, theta_ptr))


def jtrlan_mlp_set_params(net, theta_ptr):
    _check(load().jtrlan_mlp_set_params(net, theta_ptr))


def jtrlan_mlp_forward(net, x_ptr: int, N: int, y_ptr: int):
    _check(load().jtrlan_mlp_forward(net, ctypes.c_void_p(x_ptr), int(N), ctypes.c_void_p(y_ptr)))


def jtrlan_mlp_gradient(net, x_ptr: int, t_ptr: int, N: int, grad_ptr) -> float:
    loss = ctypes.c_double()
    _check(load().jtrlan_mlp_gradient(net, ctypes.c_void_p(x_ptr), ctypes.c_void_p(t_ptr), int(N), grad_ptr,
                                      ctypes.byref(loss)))
    return loss.value


def jtrlan_mlp_train(net, x_ptr: int, t_ptr: int, N: int, steps: int, lr: float, hist_ptr):
    _check(load().jtrlan_mlp_train(net, ctypes.c_void_p(x_ptr), ctypes.c_void_p(t_ptr), int(N), int(steps),
                                   ctypes.c_float(lr), hist_ptr))


def jtrlan_mlp_destroy(net):
    if net:
        load().jtrlan_mlp_destroy(net)


# ---------------------------------------------------------------- builders for the structs
def stencil_operator(dims, m0, kappa, U_ptr, W_ptr, dtype=JTRLAN_C128) -> jtrlan_operator:
    op = jtrlan_operator()
    op.kind, op.dtype = JTRLAN_STENCIL4D, dtype
    vol = int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])
    op.n = 6 * vol
    for d in range(4):
        op.dims[d] = int(dims[d])
    op.m0, op.kappa = float(m0), float(kappa)
    op.U, op.W = U_ptr, W_ptr
    return op


def dense_operator(n, a11_ptr, a12_ptr, dtype=JTRLAN_C128) -> jtrlan_operator:
    op = jtrlan_operator()
    op.kind, op.dtype, op.n = JTRLAN_DENSE, dtype, int(n)
    op.a11, op.a12 = a11_ptr, a12_ptr
    return op


def params(nev, m, mwin, tol, which=JTRLAN_SMALLEST, precision=JTRLAN_FP64, max_restarts=0,
           gs_max_passes=0, v1_ptr=None, check_jsym=0, profile=0, filter_coeffs=None, filter_window=None,
           filter_final_coeffs=None, plain_trlan=0, rotate_simt=0, invert=0, cg_tol=0.0,
           cg_max_iter=0, gs_split=0) -> jtrlan_params:
    """filter_coeffs / filter_final_coeffs: float64 arrays g_0..g_d (kept alive on the struct until
    create copies them); filter_window: (lo, hi)."""
    p = jtrlan_params()
    p.nev, p.m, p.mwin, p.tol = int(nev), int(m), int(mwin), float(tol)
    p.which, p.precision = int(which), int(precision)
    p.max_restarts, p.gs_max_passes = int(max_restarts), int(gs_max_passes)
    p.v1 = v1_ptr
    p.check_jsym = int(check_jsym)
    p.profile = int(profile)
    p.plain_trlan = int(plain_trlan)
    p.rotate_simt = int(rotate_simt)
    p.invert, p.cg_tol, p.cg_max_iter = int(invert), float(cg_tol), int(cg_max_iter)
    p.gs_split = int(gs_split)
    if filter_coeffs is not None:
        import numpy as np
        g = np.ascontiguousarray(filter_coeffs, dtype=np.float64)
        p._filter_keep = g
        p.filter_degree = len(g) - 1
        p.filter_coeffs = g.ctypes.data
        p.filter_lo, p.filter_hi = float(filter_window[0]), float(filter_window[1])
    if filter_final_coeffs is not None:
        import numpy as np
        g2 = np.ascontiguousarray(filter_final_coeffs, dtype=np.float64)
        p._filter_final_keep = g2
        p.filter_final_degree = len(g2) - 1
        p.filter_final_coeffs = g2.ctypes.data
        p.filter_lo, p.filter_hi = float(filter_window[0]), float(filter_window[1])
    return p
