"""Cyclic Jacobi eigensolver for real symmetric matrices, FP64 (oracle, test-only).

Algorithm 1 needs the eigendecomposition T_m = Z Lambda Z^T of the real symmetric
T-bar; the paper leaves the method open.  The oracle uses the textbook cyclic-by-row
Jacobi method (Jacobi 1846; Golub & Van Loan, "Matrix Computations", Sec. 8.5): sweep
over the off-diagonal pairs (p, q), p < q, in row order; for each, the rotation
J(p, q, theta) that zeroes a_pq is taken from the 2 x 2 symmetric Schur decomposition

    tau = (a_qq - a_pp) / (2 a_pq),  t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
    c = 1 / sqrt(1 + t^2),  s = t c,

and applied as A := J^T A J, Z := Z J.  Sweeps stop once off(A) = ||A - diag(A)||_F is
below eps * ||A||_F.  Each rotation is applied to whole rows and columns with numpy
vector operations; nothing is blocked or reordered.
"""
from __future__ import annotations

import numpy as np


def jacobi_eigh(T, eps=1e-15, max_sweeps=60):
    """(lam, Z) with T = Z diag(lam) Z^T, Z orthogonal, lam ascending (ties in index order)."""
    A = np.array(T, dtype=np.float64, copy=True)
    m = A.shape[0]
    if A.shape != (m, m):
        raise ValueError("square matrix expected")
    Z = np.eye(m)
    if m == 1:
        return A.diagonal().copy(), Z
    norm = np.linalg.norm(A)
    for _ in range(max_sweeps):
        off = np.linalg.norm(A - np.diag(A.diagonal()))   # formed directly, not as a difference
        if off <= eps * norm:
            break
        for p in range(m - 1):
            for q in range(p + 1, m):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                tau = (A[q, q] - A[p, p]) / (2.0 * apq)
                if abs(tau) > 1e150:       # tau^2 would overflow; t -> 1/(2 tau) in that limit
                    t = 0.5 / tau
                else:
                    t = (1.0 if tau >= 0.0 else -1.0) / (abs(tau) + np.sqrt(1.0 + tau * tau))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                # A := J^T A J with J the identity except J[p,p] = J[q,q] = c, J[p,q] = s, J[q,p] = -s
                ap, aq = A[:, p].copy(), A[:, q].copy()
                A[:, p] = c * ap - s * aq
                A[:, q] = s * ap + c * aq
                ap, aq = A[p, :].copy(), A[q, :].copy()
                A[p, :] = c * ap - s * aq
                A[q, :] = s * ap + c * aq
                A[p, q] = A[q, p] = 0.0
                zp, zq = Z[:, p].copy(), Z[:, q].copy()
                Z[:, p] = c * zp - s * zq
                Z[:, q] = s * zp + c * zq
    else:
        raise RuntimeError("Jacobi did not converge")
    lam = A.diagonal().copy()
    order = np.argsort(lam, kind="stable")
    return lam[order], Z[:, order]
