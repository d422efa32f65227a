"""TRLAN-JSYM (Algorithm 1) and LANCZOS_JSYM (Algorithm 2) in plain FP64 numpy (oracle, test-only).

Written from Sec. 3 of Ishikawa & Sogabe in the paper's order and notation.  Indices
are 0-based here: column j of V is the paper's v_{j+1}.  W = J V* is formed column by
column where Algorithm 2 uses it, exactly as the paper states it.

Readings where the paper is silent or ambiguous:

R1  Algorithm 2 divides by b0 after its Gram-Schmidt loop; on exit b0 still holds the
    norm before the last pass.  We normalise by the norm after the last pass (b1)
    and store it as t_{j+1,j}, so that V^H V = I and eq. (6) hold.
R2  t_{j,j} = v_j^H A v_j is real in exact arithmetic (Sec. 2); we keep its real part.
R4  The Gram-Schmidt loop has no cap in the paper; we stop after ``gs_max_passes``
    passes (3) and keep the last norm.
R5  Breakdown (beta below ``breakdown_tol`` times the largest |t|) is excluded by the
    paper's assumption; we raise BreakdownError.
R6  is_convd(i) is reset to false at the start of every outer iteration.
R7  The sort that moves converged pairs to the top is stable and acts on the first
    nev positions; the final output is sorted by eigenvalue (ascending for
    'smallest', descending for 'largest').
R9  v_1 = (1, ..., 1)/sqrt(n) as in Algorithm 1 unless a start vector is given.
R13 The eigendecomposition T_m = Z Lambda Z^T, for which the paper names no method, is the
    oracle's own cyclic Jacobi (jacobi.py).
R20 Invert mode (Algorithm 1's second branch): the Lanczos product is A^{-1} v_j, given as the
    function ``solve``; the wanted Ritz values of T are its largest (A's smallest); every restart
    takes c = ||A v_{m+1}|| with v_{m+1} the last Lanczos vector, and ev(i) = 1/lambda_i,
    res_est(i) = c |t_{m+1,i} ev(i)|.  The true residuals use A (``matvec``).
"""
from __future__ import annotations

import numpy as np

from .jacobi import jacobi_eigh
from .jsym import pair


class BreakdownError(RuntimeError):
    pass


class NoConvergenceError(RuntimeError):
    pass


def lanczos_jsym(matvec, V, T, k, m, gamma=np.sqrt(2.0), gs_max_passes=3,
                 breakdown_tol=1e-14, stats=None, use_w=True):
    """Algorithm 2: extend V[:, :k+1], T[:k+1, :k+1] to V[:, :m+1], T[:m+1, :m] (in place).

    ``T`` is the (m+1) x (m+1) real array holding T-bar; it is kept symmetric in its
    leading m x m part, and row m holds t_{m+1, m} = beta_m.

    With use_w=False this is the Lanczos step of the standard TRLAN, which the paper obtains
    by removing W from Algorithms 1 and 2 (Sec. 3).
    """
    for j in range(k, m):
        vj = V[:, j]
        y = matvec(vj)                                   # v_{j+1} = A v_j
        if stats is not None:
            stats["n_matvec"] += 1
        t_jj = np.vdot(vj, y).real                       # t_{j,j} = v_j^H v_{j+1}  (R2)
        T[j, j] = t_jj
        y = y - vj * t_jj                                # v_{j+1} -= v_j t_{j,j}
        b0 = np.linalg.norm(y)
        b1 = b0
        for _ in range(gs_max_passes):                   # the reorthogonalisation loop (R4)
            for i in range(j + 1):
                if use_w:
                    wi = pair(V[:, i])                   # w_i = J v_i^*
                    c = np.vdot(wi, y)
                    y = y - wi * c                       # orthogonalise against W_j
                vi = V[:, i]
                c = np.vdot(vi, y)
                y = y - vi * c                           # ... and against V_j
            if stats is not None:
                stats["n_gs_passes"] += 1
            b1 = np.linalg.norm(y)
            if b1 * gamma > b0:
                break
            b0 = b1
        beta = b1                                        # R1
        scale = max(np.max(np.abs(T[:j + 1, :j + 1])), 1.0)
        if beta <= breakdown_tol * scale:
            raise BreakdownError(f"Lanczos breakdown at step {j + 1}: beta={beta:.3e}")
        V[:, j + 1] = y / beta                           # v_{j+1} := v_{j+1} / b
        T[j + 1, j] = beta                               # t_{j+1,j} = b
        if j + 1 < m:
            T[j, j + 1] = beta
        # w_{j+1} = J v_{j+1}^* is never stored: pair() forms it where it is used.


def trlan_jsym(matvec, n, nev, m, mwin, tol, which="smallest", v1=None, max_restarts=1000,
               gs_max_passes=3, on_lanczos=None, use_w=True, solve=None):
    """Algorithm 1 (TRLAN-JSYM), normal mode; invert mode when ``solve`` (b -> A^{-1} b) is given
    (which must then be 'smallest', R20).

    Returns a dict with ``evals`` (nev,), ``X`` (n, nev), ``res`` (nev,), and the
    counters ``n_matvec`` (as counted in Sec. 3: the Lanczos-step products only),
    ``n_resid_matvec``, ``n_restarts`` (N_conv) and ``n_gs_passes``.

    ``on_lanczos(V, T, k, m)`` is called after every Lanczos phase (for invariant tests).
    """
    if n % 2 or not (0 < nev < m) or mwin < 0 or m >= n // 2:
        raise ValueError("need even n, 0 < nev < m < n/2 and mwin >= 0")
    invert = solve is not None
    if invert and which != "smallest":
        raise ValueError("invert mode finds the smallest eigenvalues")
    largest_of_T = (which == "largest") or invert
    V = np.zeros((n, m + 1), dtype=np.complex128)
    T = np.zeros((m + 1, m + 1))
    stats = dict(n_matvec=0, n_resid_matvec=0, n_gs_passes=0, n_restarts=0)
    k = 0
    v = np.ones(n, dtype=np.complex128) if v1 is None else np.asarray(v1, dtype=np.complex128).copy()
    V[:, 0] = v / np.linalg.norm(v)                      # v_1 = 1 / ||1||   (R9)
    ev = np.zeros(nev)
    res = np.full(nev, np.inf)
    res_est = np.full(nev, np.inf)
    history = []
    for _ in range(max_restarts):
        lanczos_jsym(solve if invert else matvec, V, T, k, m, gs_max_passes=gs_max_passes, stats=stats,
                     use_w=use_w)
        stats["n_restarts"] += 1
        if on_lanczos is not None:
            on_lanczos(V, T, k, m)
        beta_m = T[m, m - 1]
        lam, Z = jacobi_eigh(T[:m, :m])                  # T_m = Z Lambda Z^T (cyclic Jacobi, R13)
        order = np.argsort(-lam if largest_of_T else lam, kind="stable")
        lam, Z = lam[order], Z[:, order]                 # desired pairs first
        V[:, :m] = V[:, :m] @ Z                          # V_m := V_m Z_m
        T[:, :] = 0.0                                    # Krylov-Schur form of T-bar
        for i in range(m):
            T[i, i] = lam[i]
            T[m, i] = beta_m * Z[m - 1, i]               # t_{m+1,i} = t_{m+1,m} z_{m,i}
        if invert:                                       # R20
            c = np.linalg.norm(matvec(V[:, m]))          # c = ||A v_{m+1}||
            stats["n_resid_matvec"] += 1
            ev = 1.0 / lam[:nev]
            res_est = c * np.abs(T[m, :nev] * ev)
        else:
            ev = lam[:nev].copy()
            res_est = np.abs(T[m, :nev]).copy()
        is_convd = np.zeros(nev, dtype=bool)             # R6
        for i in range(nev):
            if res_est[i] < tol:                         # check the true residual
                r = matvec(V[:, i]) - V[:, i] * ev[i]
                stats["n_resid_matvec"] += 1
                res[i] = np.linalg.norm(r)
                is_convd[i] = res[i] < tol
        # move converged pairs to the top (stable sort on the key is_convd)   (R7)
        perm = np.concatenate([np.flatnonzero(is_convd), np.flatnonzero(~is_convd)])
        V[:, :nev] = V[:, perm]
        Z[:, :nev] = Z[:, perm]
        lam[:nev] = lam[perm]
        T[m, :nev] = T[m, perm]
        for i in range(nev):
            T[i, i] = lam[i]
        res, res_est, ev, is_convd = res[perm], res_est[perm], ev[perm], is_convd[perm]
        icnv = 0
        for i in range(nev):
            if is_convd[i]:
                T[m, i] = 0.0                            # decouple the converged subspace
                icnv += 1
        history.append(dict(ev=ev.copy(), res_est=res_est.copy(), icnv=icnv))
        if icnv == nev:
            break
        k = min(icnv + mwin, m - 1)                      # eq. (29)
        arrow = T[m, :k].copy()
        T[k + 1:, :] = 0.0
        T[:, k + 1:] = 0.0
        T[k, :] = 0.0
        T[k, :k] = arrow                                 # t_{k+1,i} = t_{m+1,i}
        T[:k, k] = arrow
        V[:, k] = V[:, m]                                # v_{k+1} = v_{m+1}
        # W_{k+1} = J V_{k+1}^* is implicit (pair() forms it on use)
    else:
        raise NoConvergenceError(f"not converged after {max_restarts} restarts")
    order = np.argsort(ev if which == "smallest" else -ev, kind="stable")
    return dict(evals=ev[order], X=V[:, :nev][:, order].copy(), res=res[order],
                history=history, **stats)
