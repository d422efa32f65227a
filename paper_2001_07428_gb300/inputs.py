"""Seeded synthetic inputs for J-TRLan (shared by tests, bench and the oracle's callers).

This module only draws random numbers and lays them out; it contains none of the
eigensolver's arithmetic and imports nothing else from this package.  Both the
CUDA path and the CPU oracle receive the arrays it returns.

Layouts (the library's canonical layout):

* dense operator: ``A11`` and ``A12`` are (h, h) complex row-major with h = n/2
  (the blocks of the Hermitian J-symmetric form, Sec. 1 eq. (4)).
* stencil operator on a periodic lattice ``dims = (Lx, Ly, Lz, Lt)``: the site index
  is ``s = x + Lx*(y + Ly*(z + Lz*t))`` (x fastest); the link fields ``U`` and ``W``
  are (4, V, 3, 3) complex row-major, direction mu = 0..3 along x, y, z, t.
* vectors: length n = 2*h; the first half holds x1, the second x2; for the
  stencil h = 3*V and element ``3*s + colour`` of each half.
"""
from __future__ import annotations

import numpy as np


def complex_gaussian(rng: np.random.Generator, shape) -> np.ndarray:
    """Complex Gaussian with independent N(0,1) real and imaginary parts."""
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def dense_jsym(h: int, seed: int):
    """Dense Hermitian J-symmetric blocks: A11 = (G+G^H)/2, A12 = (K-K^T)/2.

    G and K are complex Gaussian (h, h).  Returns (A11, A12) as complex128.
    """
    rng = np.random.default_rng(seed)
    G = complex_gaussian(rng, (h, h))
    K = complex_gaussian(rng, (h, h))
    A11 = 0.5 * (G + G.conj().T)
    A12 = 0.5 * (K - K.T)
    return np.ascontiguousarray(A11), np.ascontiguousarray(A12)


def haar_su3(rng: np.random.Generator, count: int) -> np.ndarray:
    """``count`` Haar-random SU(3) matrices, shape (count, 3, 3) complex128.

    QR of a complex Gaussian matrix with the diagonal phases of R moved into Q
    (Mezzadri 2007) gives Haar U(3); dividing by the principal cube root of the
    determinant maps it to SU(3) and keeps the Haar measure.
    """
    Zm = complex_gaussian(rng, (count, 3, 3)) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Zm)
    d = np.diagonal(R, axis1=1, axis2=2)
    ph = d / np.abs(d)
    Q = Q * ph[:, None, :]
    det = np.linalg.det(Q)
    root = np.exp(1j * np.angle(det) / 3.0)
    return Q / root[:, None, None]


def lattice_volume(dims) -> int:
    return int(np.prod([int(d) for d in dims]))


def stencil_links(dims, seed: int):
    """Random links: U Haar SU(3) per (mu, site), W complex Gaussian 3x3 per (mu, site)."""
    V = lattice_volume(dims)
    rng = np.random.default_rng(seed)
    U = haar_su3(rng, 4 * V).reshape(4, V, 3, 3)
    W = complex_gaussian(rng, (4, V, 3, 3))
    return np.ascontiguousarray(U), np.ascontiguousarray(W)


def constant_links(dims, seed: int):
    """Translation-invariant links: one U_mu (SU(3)) and one W_mu (Gaussian) per direction."""
    V = lattice_volume(dims)
    rng = np.random.default_rng(seed)
    U0 = haar_su3(rng, 4)
    W0 = complex_gaussian(rng, (4, 3, 3))
    U = np.broadcast_to(U0[:, None], (4, V, 3, 3)).copy()
    W = np.broadcast_to(W0[:, None], (4, V, 3, 3)).copy()
    return U, W, U0, W0


def free_links(dims):
    """Unit gauge links and W = 0 (the free field)."""
    V = lattice_volume(dims)
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, V, 3, 3)).copy()
    W = np.zeros((4, V, 3, 3), dtype=np.complex128)
    return U, W


def case_a(n: int, seed: int):
    """A random Hermitian J-symmetric matrix in the diagonal block form A = U diag(L, L) U^H,
    U = [[X1, -X2^*], [X2, X1^*]] (Sec. 4, Case A): L uniform in (0, 1); X1, X2 entries uniform in
    the box (-1, 1) + i(-1, 1), then made to satisfy X1^H X1 + X2^H X2 = I and X1^T X2 - X2^T X1 = O
    by Gram-Schmidt against the columns of X and of J X^* (two passes, in blocks of 50 columns).
    Returns (A11, A12, L): the blocks of the block form (eq. (4)) and the n/2 eigenvalues."""
    h = n // 2
    rng = np.random.default_rng(seed)
    lam = rng.uniform(0.0, 1.0, h)
    X = rng.uniform(-1, 1, (n, h)) + 1j * rng.uniform(-1, 1, (n, h))

    def jstar(Y):            # columns J y^* with J = [[O, -I], [I, O]]
        return np.concatenate([-np.conj(Y[h:]), np.conj(Y[:h])], axis=0)

    done = 0
    while done < h:
        b = min(50, h - done)
        blk = X[:, done:done + b]
        for _ in range(2):   # against the finished columns and their partners
            if done:
                Q = X[:, :done]
                blk = blk - Q @ (Q.conj().T @ blk)
                P = jstar(Q)
                blk = blk - P @ (P.conj().T @ blk)
        for c in range(b):   # within the block, column by column
            x = blk[:, c]
            for _ in range(2):
                if c:
                    Q = blk[:, :c]
                    x = x - Q @ (Q.conj().T @ x)
                    P = jstar(Q)
                    x = x - P @ (P.conj().T @ x)
            blk[:, c] = x / np.linalg.norm(x)
        X[:, done:done + b] = blk
        done += b
    U = np.concatenate([X, jstar(X)], axis=1)
    A = (U * np.concatenate([lam, lam])) @ U.conj().T
    return np.ascontiguousarray(A[:h, :h]), np.ascontiguousarray(A[:h, h:]), lam


def random_vector(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return complex_gaussian(rng, (n,))


def batched_dense_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Even sizes drawn uniformly from {lo, lo+2, ..., hi}."""
    rng = np.random.default_rng(seed)
    return 2 * rng.integers(lo // 2, hi // 2 + 1, size=count)


# The workloads (sizes, seeds, solver parameters).  mwin follows the paper's habit
# mwin = 2*nev capped at m/2 where a workload does not state it.
WORKLOADS = {
    "dense_n200": dict(kind="dense", n=200, seed=0, nev=10, m=30, mwin=15),
    "stencil_8x8x8x8": dict(kind="stencil", dims=(8, 8, 8, 8), m0=8.5, kappa=0.3, seed=1,
                            nev=20, m=60, mwin=30),
    "stencil_16x16x16x16": dict(kind="stencil", dims=(16, 16, 16, 16), m0=8.5, kappa=0.3, seed=1,
                                nev=50, m=120, mwin=60),
    # the largest lattice: links stored in complex64, as its workload states
    "stencil_24x24x24x48": dict(kind="stencil", dims=(24, 24, 24, 48), m0=8.5, kappa=0.3, seed=1,
                                nev=100, m=200, mwin=100, links="c64"),
}
