"""Convenience layer over the C ABI for PyTorch users: uploads arrays, calls jtrlan_create /
jtrlan_solve / jtrlan_pairs, and returns torch tensors.  Marshalling only; the solve runs in
libjtrlan's kernels on the current CUDA stream."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import binding as B


def _dev(a, device):
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=torch.complex128).contiguous()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to(device)


class JTRLan:
    """One operator + parameter set bound to a library context on ``device``.

    ``kind`` is "stencil" (U, W of shape (4, V, 3, 3), dims, m0, kappa) or "dense" (A11, A12).
    """

    def __init__(self, kind, *, nev, m, mwin, tol, which="smallest", dims=None, m0=None, kappa=None,
                 U=None, W=None, A11=None, A12=None, v1=None, max_restarts=0, gs_max_passes=0,
                 check_jsym=False, profile=False, precision="fp64", filter_coeffs=None, filter_window=None,
                 filter_final_coeffs=None, plain_trlan=False, links_dtype="c128", rotate_simt=False,
                 invert=False, cg_tol=0.0, cg_max_iter=0, gs_split=False, device="cuda"):
        B.load()
        self.device = torch.device(device)
        self.stream = torch.cuda.current_stream(self.device)
        keep = []
        if kind == "stencil":
            Ud, Wd = _dev(U, self.device), _dev(W, self.device)
            dt = B.JTRLAN_C128
            if links_dtype == "c64":
                Ud, Wd, dt = Ud.to(torch.complex64), Wd.to(torch.complex64), B.JTRLAN_C64
            keep += [Ud, Wd]
            op = B.stencil_operator(dims, m0, kappa, Ud.data_ptr(), Wd.data_ptr(), dtype=dt)
        elif kind == "dense":
            Ad, Bd = _dev(A11, self.device), _dev(A12, self.device)
            keep += [Ad, Bd]
            op = B.dense_operator(2 * Ad.shape[0], Ad.data_ptr(), Bd.data_ptr())
        else:
            raise ValueError(kind)
        self.n = int(op.n)
        self.nev = int(nev)
        v1p = None
        if v1 is not None:
            v1d = _dev(v1, self.device)
            keep.append(v1d)
            v1p = v1d.data_ptr()
        w = B.JTRLAN_LARGEST if which == "largest" else B.JTRLAN_SMALLEST
        self._keep_v1 = keep[-1] if v1 is not None else None
        prec = {"fp64": B.JTRLAN_FP64, "mixed": B.JTRLAN_MIXED, "mixed_reorth": B.JTRLAN_MIXED_REORTH}[precision]
        self.mixed = prec != B.JTRLAN_FP64
        self.fp32_filter = prec == B.JTRLAN_MIXED and filter_coeffs is not None and len(filter_coeffs) > 1
        prm = B.params(nev, m, mwin, tol, which=w, precision=prec, max_restarts=max_restarts,
                       gs_max_passes=gs_max_passes, v1_ptr=v1p, check_jsym=int(check_jsym),
                       profile=int(profile), filter_coeffs=filter_coeffs, filter_window=filter_window,
                       filter_final_coeffs=filter_final_coeffs, plain_trlan=int(plain_trlan),
                       rotate_simt=int(rotate_simt), invert=int(invert), cg_tol=cg_tol,
                       cg_max_iter=cg_max_iter, gs_split=int(gs_split))
        self.ctx = B.jtrlan_create(op, prm, self.stream.cuda_stream)
        # jtrlan_create copied the operator; v1 is read at solve time, so it is kept alive.

    def apply(self, x: torch.Tensor) -> torch.Tensor:
        """y = A x: complex128 for an FP64 context, complex64 (the FP32 operator) for a mixed one."""
        x = _dev(x, self.device)
        if self.mixed:
            x = x.to(torch.complex64)
        y = torch.empty_like(x)
        B.jtrlan_apply(self.ctx, x.data_ptr(), y.data_ptr())
        return y

    def solve(self) -> dict:
        return B.jtrlan_solve(self.ctx)

    def pairs(self, with_partners=False):
        ev = np.zeros(self.nev)
        res = np.zeros(self.nev)
        ncol = 2 * self.nev if with_partners else self.nev
        X = torch.empty((ncol, self.n), dtype=torch.complex128, device=self.device)
        B.jtrlan_pairs(self.ctx, int(with_partners), ev.ctypes.data_as(ctypes.c_void_p),
                       ctypes.c_void_p(X.data_ptr()), res.ctypes.data_as(ctypes.c_void_p))
        return ev, X.T, res   # X.T is n x ncol (column-major storage)

    def profile(self) -> dict:
        return B.jtrlan_get_profile(self.ctx)

    def apply_filter(self, x: torch.Tensor) -> torch.Tensor:
        """y = p(A) x with the context's filter: the FP32-phase filter and FP32 operator (complex64) where
        the context has one, else the certifying filter with the solve's own product (complex128)."""
        x = _dev(x, self.device)
        if self.fp32_filter:
            x = x.to(torch.complex64)
        y = torch.empty_like(x)
        B.jtrlan_apply_filter(self.ctx, x.data_ptr(), y.data_ptr())
        return y

    def bounds(self, steps=20):
        """(lo, hi): spectral window estimate from `steps` unrestarted Lanczos steps (jtrlan_bounds)."""
        return B.jtrlan_bounds(self.ctx, steps)

    def close(self):
        if getattr(self, "ctx", None):
            B.jtrlan_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class JTRLanBatch:
    """Many dense operators (lists of A11, A12 blocks of uneven order) solved in one persistent launch.

    ``precision`` is "fp64" or "mixed_reorth" (compensated FP32 products and Gram-Schmidt).
    """

    def __init__(self, A11s, A12s, *, nev, m, mwin, tol, which="smallest", max_restarts=0, gs_max_passes=0,
                 precision="fp64", profile=False, device="cuda"):
        B.load()
        self.device = torch.device(device)
        self.stream = torch.cuda.current_stream(self.device)
        blocks = [(_dev(a, self.device), _dev(b, self.device)) for a, b in zip(A11s, A12s)]
        ops = [B.dense_operator(2 * a.shape[0], a.data_ptr(), b.data_ptr()) for a, b in blocks]
        self.ns = [int(o.n) for o in ops]
        self.nev = int(nev)
        w = B.JTRLAN_LARGEST if which == "largest" else B.JTRLAN_SMALLEST
        prec = {"fp64": B.JTRLAN_FP64, "mixed_reorth": B.JTRLAN_MIXED_REORTH}[precision]
        prm = B.params(nev, m, mwin, tol, which=w, precision=prec, max_restarts=max_restarts,
                       gs_max_passes=gs_max_passes, profile=int(profile))
        self.b = B.jtrlan_batch_create(ops, prm, self.stream.cuda_stream)
        # jtrlan_batch_create copied the blocks and synchronised; they may be released now.

    def tune(self) -> dict:
        return B.jtrlan_batch_tune(self.b)

    def set_shape(self, threads, ctas_per_sm=0):
        B.jtrlan_batch_set_shape(self.b, threads, ctas_per_sm)

    def set_tiles(self, mv_rows, gs_groups=0):
        B.jtrlan_batch_set_tiles(self.b, mv_rows, gs_groups)

    def solve(self, check=True) -> dict:
        return B.jtrlan_batch_solve(self.b, check=check)

    def results(self):
        """(evals, res, istats): (count, nev), (count, nev), (count, 6) numpy arrays; istats columns:
        Lanczos products, outer iterations, status, residual products, Ritz fallbacks, GS passes."""
        cnt = len(self.ns)
        ev = np.zeros((cnt, self.nev))
        res = np.zeros((cnt, self.nev))
        ist = np.zeros((cnt, B.BATCH_STATS), dtype=np.int32)
        B.jtrlan_batch_results(self.b, ev.ctypes.data_as(ctypes.c_void_p), res.ctypes.data_as(ctypes.c_void_p),
                               ist.ctypes.data_as(ctypes.c_void_p))
        return ev, res, ist

    def vectors(self, i) -> torch.Tensor:
        X = torch.empty((self.nev, self.ns[i]), dtype=torch.complex128, device=self.device)
        B.jtrlan_batch_vectors(self.b, i, ctypes.c_void_p(X.data_ptr()))
        return X.T   # n_i x nev

    def close(self):
        if getattr(self, "b", None):
            B.jtrlan_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
