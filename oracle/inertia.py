"""Eigenvalue counts by Sylvester's law of inertia (oracle, test-only).

For a Hermitian matrix A and a real shift sigma, the number of eigenvalues of A below sigma equals the
number of negative eigenvalues of D in any factorisation A - sigma I = L D L^H with L nonsingular
(Sylvester's law of inertia).  The factorisation is LAPACK's Bunch-Kaufman LDL^H (zhetrf, through
scipy.linalg.ldl): D is block diagonal with 1x1 and 2x2 Hermitian blocks, whose eigenvalues are
counted directly.

This is what the paper's method cannot give by itself: Algorithm 1 returns nev converged pairs, not a
proof that no eigenvalue below them was missed.  A count below a shift placed between the found
lambda_nev and the next eigenvalue closes that gap; for a Hermitian J-symmetric A every eigenvalue is
doubly degenerate (eq. (2)), so the count is 2 nev.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def count_below(A: np.ndarray, sigma: float, overwrite: bool = False) -> int:
    """Number of eigenvalues of the Hermitian matrix A below sigma (LDL^H inertia of A - sigma I)."""
    M = A if overwrite else np.array(A, copy=True)
    M[np.diag_indices_from(M)] -= sigma
    _, d, _ = scipy.linalg.ldl(M, lower=True, hermitian=True, overwrite_a=True, check_finite=False)
    neg = 0
    i, n = 0, d.shape[0]
    while i < n:
        if i + 1 < n and d[i + 1, i] != 0:          # a 2x2 block [[a, conj(b)], [b, c]]
            blk = np.array([[d[i, i], d[i, i + 1]], [d[i + 1, i], d[i + 1, i + 1]]])
            neg += int((np.linalg.eigvalsh(blk) < 0).sum())
            i += 2
        else:
            neg += int(d[i, i].real < 0)
            i += 1
    return neg
