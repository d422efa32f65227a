"""Conjugate gradients in plain FP64 numpy (oracle, test-only).

The inner solver of Algorithm 1's invert mode (Sec. 4 solves A x = v_j with CG).  This is the
Hestenes-Stiefel iteration written from its textbook definition for a Hermitian positive definite
operator given as a function:

    x_0 = 0, r_0 = b, p_0 = r_0
    alpha_k = (r_k^H r_k) / (p_k^H A p_k)
    x_{k+1} = x_k + alpha_k p_k,   r_{k+1} = r_k - alpha_k A p_k
    beta_k = (r_{k+1}^H r_{k+1}) / (r_k^H r_k),   p_{k+1} = r_{k+1} + beta_k p_k

stopping once ||r_k|| <= rtol ||b||.
"""
from __future__ import annotations

import numpy as np


class NotPositiveDefiniteError(RuntimeError):
    pass


def cg(matvec, b, rtol=1e-12, max_iter=10000, history=None):
    """Returns (x, iterations).  ``history`` (a list) receives every iterate x_k if given."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    stop = (rtol ** 2) * rr
    if history is not None:
        history.append(x.copy())
    if rr == 0.0:
        return x, 0
    for k in range(1, max_iter + 1):
        q = matvec(p)
        pap = np.vdot(p, q).real
        if not pap > 0.0:
            raise NotPositiveDefiniteError("p^H A p <= 0")
        alpha = rr / pap
        x = x + alpha * p
        r = r - alpha * q
        rr_new = np.vdot(r, r).real
        if history is not None:
            history.append(x.copy())
        if rr_new <= stop:
            return x, k
        p = r + (rr_new / rr) * p
        rr = rr_new
    raise RuntimeError(f"CG did not converge in {max_iter} iterations")
