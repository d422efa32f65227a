"""The learned polynomial filter for the stencil operator (the paper has no filter).

A 3-layer perceptron (width 128, FP32; the library's jtrlan_mlp_* kernels) maps cheap features of a
problem -- the spectral window estimated by jtrlan_bounds, the lattice parameters m0 and kappa, and
nev -- to the DEGREE + 1 Chebyshev coefficients g_0..g_DEGREE of a real filter p on that window.  The
solver (JTRLAN_MIXED_REORTH: FP64 vectors, compensated-FP32 products and Gram-Schmidt) runs Algorithm 1
on B = p(A) and accepts a pair only when the true residual of A at x^H A x is below tol, so the plain
method's criterion judges every answer, and the unfiltered solve is the fallback (solve_learned reruns
it if the filtered solve fails).  Degree 64, the most allowed, was the fastest of 16, 24, 32, 48 and
64 on the 24^3 x 48 lattice (nev 100, m 200): a sharper step separates the dense wanted cluster in
fewer Lanczos steps, and each step's Gram-Schmidt against up to 200 columns costs more than the extra
products.  A filter of lower degree with the same cut is one call away (at_degree).

Training targets come from plain runs of the method: lambda_nev places the cut CUT_OFFSET transition
widths below it, and the Jackson-damped step (jtrlan_damped_step) with that cut is the target.  The
solver takes the exact damped step at the cut the network predicts (at_degree).

Everything here is marshalling and bookkeeping on a few scalars per problem; every vector operation,
the network and its training run in the library's kernels.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np
import torch

from . import binding as B

PKG = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(PKG, "filter_mlp.npz")
RUNS = os.path.join(PKG, "filter_runs.json")   # the plain runs the network was trained on
DEGREE = 64
WIDTH = 128
N_FEATURES = 5
BOUNDS_STEPS = 30
NEV_GRID = (8, 10, 12, 16, 20, 25, 30, 40, 50, 60, 70, 80, 90, 100)


def window(lo: float, hi: float):
    """The filter window [a, b]: the bounds estimate widened by 2% below (lo is an estimate)."""
    return lo - 0.02 * (hi - lo), hi


def features(lo, hi, m0, kappa, nev, sites) -> np.ndarray:
    """Five O(1) inputs of the network: the bounds, the lattice parameters, and the wanted fraction
    nev/sites of the spectrum (the cut follows the integrated density of states at that fraction; nev
    alone is left out, so that a large lattice with many wanted pairs interpolates between smaller
    lattices at the same fraction instead of extrapolating)."""
    return np.array([(lo - m0) / 8.0, (hi - m0) / 8.0, m0 - 9.0, (kappa - 0.3) / 0.2,
                     np.log(nev / sites) / 3.0 + 2.0], dtype=np.float32)


# Where the filter's step sits, in units of its transition width pi/DEGREE (in theta = arccos of the
# window coordinate): CUT_OFFSET widths below lambda_nev, so that the wanted eigenvalues lie in the
# steep lower tail of the damped step, where p falls by a large factor from each wanted eigenvalue to
# the next (relative gaps in the spectrum of B = p(A) are what Lanczos resolves).  Measured on GB300
# with the step moved over offsets 1.5, 2, 2.5, 3 (24^3 x 48, nev 100: 13.7, 12.2, 16.8, 206 s; the
# midpoint between lambda_nev and lambda_{nev+1}: 22.5 s): 2 was the fastest, or within 2% of it, on
# 8^4 (nev 20), 12^4 (nev 30 and 100), 16^4 (nev 50) and 24^3 x 48; near 3 a ripple of the damped step
# meets the wanted set and the solve slows by 5-17x.  The target is 1.75 widths: within a few percent
# of the fastest, and a quarter width further from that cliff than the prediction error allows.
CUT_OFFSET = 1.75


def cut_tau(ev_sorted, nev, a, b) -> float:
    """Window coordinate tau of the step for a problem whose lowest eigenvalues are ev_sorted: theta =
    arccos((lambda_nev - c)/e) + CUT_OFFSET pi / DEGREE, tau = cos(theta), kept inside (-1, 1)."""
    c, e = 0.5 * (a + b), 0.5 * (b - a)
    t_nev = float(np.clip((ev_sorted[nev - 1] - c) / e, -1.0, 1.0))
    theta = min(np.arccos(t_nev) + CUT_OFFSET * np.pi / DEGREE, np.pi)
    return float(np.clip(np.cos(theta), -0.9999, 0.999))


class FilterNet:
    """The network on one device (parameters in device memory, kernels of the library)."""

    def __init__(self, theta=None, seed=0, device="cuda"):
        B.load()
        self.device = torch.device(device)
        self.stream = torch.cuda.current_stream(self.device)
        self.net = B.jtrlan_mlp_create(N_FEATURES, WIDTH, DEGREE + 1, seed, self.stream.cuda_stream)
        self.P = B.jtrlan_mlp_param_count(N_FEATURES, WIDTH, DEGREE + 1)
        if theta is not None:
            th = np.ascontiguousarray(theta, dtype=np.float32)
            assert th.size == self.P
            B.jtrlan_mlp_set_params(self.net, th.ctypes.data_as(ctypes.c_void_p))

    @classmethod
    def load(cls, path=WEIGHTS, device="cuda"):
        z = np.load(path)
        return cls(theta=z["theta"], device=device)

    def params(self) -> np.ndarray:
        th = np.zeros(self.P, dtype=np.float32)
        B.jtrlan_mlp_get_params(self.net, th.ctypes.data_as(ctypes.c_void_p))
        return th

    def save(self, path=WEIGHTS, **meta):
        np.savez(path, theta=self.params(), meta=json.dumps(meta))

    def predict(self, X: np.ndarray) -> np.ndarray:
        X = np.ascontiguousarray(np.atleast_2d(X), dtype=np.float32)
        Xd = torch.from_numpy(X).to(self.device)
        Yd = torch.empty((X.shape[0], DEGREE + 1), dtype=torch.float32, device=self.device)
        B.jtrlan_mlp_forward(self.net, Xd.data_ptr(), X.shape[0], Yd.data_ptr())
        self.stream.synchronize()
        return Yd.cpu().numpy().astype(np.float64)

    def train(self, X: np.ndarray, T: np.ndarray, steps: int, lr: float) -> np.ndarray:
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(self.device)
        Td = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).to(self.device)
        hist = np.zeros(steps, dtype=np.float32)
        B.jtrlan_mlp_train(self.net, Xd.data_ptr(), Td.data_ptr(), X.shape[0], steps, lr,
                           hist.ctypes.data_as(ctypes.c_void_p))
        return hist

    def loss(self, X: np.ndarray, T: np.ndarray) -> float:
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(self.device)
        Td = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).to(self.device)
        return B.jtrlan_mlp_gradient(self.net, Xd.data_ptr(), Td.data_ptr(), X.shape[0], None)

    def close(self):
        if getattr(self, "net", None):
            B.jtrlan_mlp_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def damped_targets(taus, device="cuda", degree=DEGREE) -> np.ndarray:
    """Jackson-damped step coefficients of the given degree for each tau, from the library kernel."""
    td = torch.from_numpy(np.ascontiguousarray(taus, dtype=np.float64)).to(device)
    out = torch.empty((len(taus), degree + 1), dtype=torch.float32, device=device)
    B.jtrlan_damped_step(td.data_ptr(), len(taus), degree, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def cut_of(coeffs) -> float:
    """The cut tau encoded by a damped step's coefficients: g_0 = (pi - acos tau)/pi."""
    return float(np.cos(np.pi * (1.0 - np.asarray(coeffs)[0])))


def at_degree(coeffs, degree, device="cuda") -> np.ndarray:
    """The Jackson-damped step of the given degree whose cut is the one the network's coefficients
    encode (g_0).  The solver always takes this exact step, not the network's raw coefficients: the
    wanted eigenvalues sit in the step's tail, where p is 1e-3 to 1e-5 and the raw outputs' error
    (about 1e-3 per coefficient) would swamp it."""
    return damped_targets([cut_of(coeffs)], device, degree)[0].astype(np.float64)


def stencil_bounds(U, W, dims, m0, kappa, device="cuda"):
    """(lo, hi) of jtrlan_bounds on the FP32 operator (BOUNDS_STEPS unrestarted Lanczos steps)."""
    from .solver import JTRLan
    s = JTRLan(kind="stencil", dims=dims, m0=m0, kappa=kappa, U=U, W=W, nev=1, m=BOUNDS_STEPS + 1, mwin=1,
               tol=1e-8, precision="mixed", device=device)
    lo, hi = s.bounds(BOUNDS_STEPS)
    s.close()
    return lo, hi


def learned_filter(net: FilterNet, U, W, dims, m0, kappa, nev, device="cuda", degree=DEGREE):
    """(coefficients, window, features) predicted for one stencil problem: the damped step at the
    network's cut (at_degree)."""
    lo, hi = stencil_bounds(U, W, dims, m0, kappa, device)
    sites = int(np.prod(dims))
    f = features(lo, hi, m0, kappa, nev, sites)
    g = at_degree(net.predict(f[None, :])[0], degree, net.device)
    return g, window(lo, hi), f


def filter_on_context(net: FilterNet, ctx, m0, kappa, nev, sites, degree=None):
    """The learned filter for the operator of an existing context, set on that context: jtrlan_bounds
    on the context itself, network inference, jtrlan_set_filter.  Returns (coefficients, window,
    features); the next jtrlan_solve of the context runs on B = p(A), p the damped step at the
    network's cut (at_degree) of the given degree (default: the network's own)."""
    lo, hi = B.jtrlan_bounds(ctx, BOUNDS_STEPS)
    f = features(lo, hi, m0, kappa, nev, sites)
    g = at_degree(net.predict(f[None, :])[0], degree or DEGREE, net.device)
    win = window(lo, hi)
    B.jtrlan_set_filter(ctx, g, win)
    return g, win, f


def solve_learned(net: FilterNet, U, W, dims, m0, kappa, nev, m, mwin, tol, device="cuda", **kw):
    """J-TRLan (JTRLAN_MIXED_REORTH) on B = p(A) with the network's filter, every pair certified by the
    true residual of A.  Falls back to the unfiltered solve if the filtered one fails.
    Returns (solver, stats, filter info)."""
    from .solver import JTRLan
    g, win, f = learned_filter(net, U, W, dims, m0, kappa, nev, device)
    base = dict(kind="stencil", dims=dims, m0=m0, kappa=kappa, U=U, W=W, nev=nev, m=m, mwin=mwin, tol=tol,
                precision="mixed_reorth", device=device, **kw)
    s = JTRLan(filter_final_coeffs=g, filter_window=win, **base)
    try:
        st = s.solve()
        return s, st, dict(coeffs=g, window=win, features=f, fallback=False)
    except B.JTRLanError:
        s.close()
        s = JTRLan(**base)
        st = s.solve()
        return s, st, dict(coeffs=g, window=win, features=f, fallback=True)
