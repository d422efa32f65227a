"""Hermitian J-symmetric operators, written from their definitions (oracle, test-only).

Paper: Ishikawa & Sogabe, "A thick-restart Lanczos type method for Hermitian
J-symmetric eigenvalue problems", Sec. 1.

* J-symmetry: J A J^{-1} = A^T with J real, J^T = -J = J^{-1}            (eq. (1))
* canonical J = [[O, -I], [I, O]] with (n/2)x(n/2) blocks                 (Sec. 1)
* pair map: if A x = lambda x then y = J x* is an eigenvector too         (eq. (2))
* block form: A = [[A11, A12], [A12^H, A11^T]], A11^H = A11, A12^T = -A12 (eq. (4))

Vectors are complex128 of even length n; the first half is x1, the second x2.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- J and the pair map
def J_matrix(n: int) -> np.ndarray:
    """The canonical J = [[O, -I], [I, O]] as a dense real matrix (Sec. 1)."""
    h = n // 2
    Jm = np.zeros((n, n))
    Jm[:h, h:] = -np.eye(h)
    Jm[h:, :h] = np.eye(h)
    return Jm


def apply_J(x: np.ndarray) -> np.ndarray:
    """J x for the canonical J: [x1; x2] -> [-x2; x1]."""
    h = x.shape[0] // 2
    return np.concatenate([-x[h:], x[:h]])


def pair(x: np.ndarray) -> np.ndarray:
    """The partner vector J x* of eq. (2)."""
    return apply_J(np.conj(x))


# ---------------------------------------------------------------- block form (eq. (4))
def assemble_block_form(A11: np.ndarray, A12: np.ndarray) -> np.ndarray:
    """Dense A = [[A11, A12], [A12^H, A11^T]] (eq. (4))."""
    return np.block([[A11, A12], [A12.conj().T, A11.T]])


def dense_matvec(A11: np.ndarray, A12: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = A x for the block form of eq. (4), one block product at a time."""
    h = A11.shape[0]
    x1, x2 = x[:h], x[h:]
    y1 = A11 @ x1 + A12 @ x2
    y2 = A12.conj().T @ x1 + A11.T @ x2
    return np.concatenate([y1, y2])


# ---------------------------------------------------------------- 4D stencil operator
# Lattice sites s = x + Lx*(y + Ly*(z + Lz*t)); reshaping a site-major array in C order
# to (Lt, Lz, Ly, Lx, ...) puts direction mu (0=x .. 3=t) on array axis 3 - mu.
def _field(a: np.ndarray, dims) -> np.ndarray:
    Lx, Ly, Lz, Lt = dims
    return a.reshape((Lt, Lz, Ly, Lx) + a.shape[1:])


def _fwd(f: np.ndarray, mu: int) -> np.ndarray:
    """f(s + mu_hat) with periodic wrap."""
    return np.roll(f, -1, axis=3 - mu)


def _bwd(f: np.ndarray, mu: int) -> np.ndarray:
    """f(s - mu_hat) with periodic wrap."""
    return np.roll(f, +1, axis=3 - mu)


def _mv(M: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Site-wise 3x3 matrix times 3-vector."""
    return np.einsum("...ab,...b->...a", M, v)


def stencil_A11(U, dims, m0, psi):
    """(A11 psi)(s) = m0 psi(s) + sum_mu [U_mu(s) psi(s+mu) + U_mu(s-mu)^H psi(s-mu)].

    This is the block A11 = m0 I + sum_mu [U_mu(x) delta_{x+mu,y} + U_mu(y)^H delta_{x-mu,y}]
    of the synthetic stencil operator.  ``psi`` is (V*3,), returns (V*3,).
    """
    V = int(np.prod(dims))
    p = _field(psi.reshape(V, 3), dims)
    out = m0 * p
    for mu in range(4):
        Uf = _field(U[mu], dims)
        out = out + _mv(Uf, _fwd(p, mu)) + _mv(np.conj(np.swapaxes(_bwd(Uf, mu), -1, -2)), _bwd(p, mu))
    return out.reshape(V * 3)


def stencil_A12(W, dims, kappa, psi):
    """(A12 psi)(s) = kappa sum_mu [W_mu(s) psi(s+mu) - W_mu(s-mu)^T psi(s-mu)].

    This is the block A12 = kappa sum_mu [W_mu(x) delta_{x+mu,y} - W_mu(y)^T delta_{x-mu,y}],
    which is skew-symmetric as eq. (4) requires.
    """
    V = int(np.prod(dims))
    p = _field(psi.reshape(V, 3), dims)
    out = np.zeros_like(p)
    for mu in range(4):
        Wf = _field(W[mu], dims)
        out = out + _mv(Wf, _fwd(p, mu)) - _mv(np.swapaxes(_bwd(Wf, mu), -1, -2), _bwd(p, mu))
    return kappa * out.reshape(V * 3)


def stencil_matvec(U, W, dims, m0, kappa, x):
    """y = A x with A = [[A11, A12], [A12^H, A11^T]] (eq. (4)) for the stencil blocks.

    The transposed and adjoint blocks are applied through conjugation:
    A11^T psi = conj(A11 conj(psi)) (A11 Hermitian) and
    A12^H psi = conj(A12^T conj(psi)) = -conj(A12 conj(psi)) (A12 skew-symmetric).
    """
    h = x.shape[0] // 2
    x1, x2 = x[:h], x[h:]
    y1 = stencil_A11(U, dims, m0, x1) + stencil_A12(W, dims, kappa, x2)
    A12H_x1 = -np.conj(stencil_A12(W, dims, kappa, np.conj(x1)))
    A11T_x2 = np.conj(stencil_A11(U, dims, m0, np.conj(x2)))
    return np.concatenate([y1, A12H_x1 + A11T_x2])


def site_index(coords, dims) -> int:
    x, y, z, t = coords
    Lx, Ly, Lz, Lt = dims
    return x + Lx * (y + Ly * (z + Lz * t))


def stencil_blocks_dense(U, W, dims, m0, kappa):
    """Dense A11 and A12 of the stencil, entry by entry from the delta-function definitions.

    Brute force for small lattices only: loops over sites and directions and adds the
    3x3 blocks [x, x+mu] and [x, x-mu] (periodic) one at a time.
    """
    dims = tuple(int(d) for d in dims)
    V = int(np.prod(dims))
    h = 3 * V
    A11 = np.zeros((h, h), dtype=np.complex128)
    A12 = np.zeros((h, h), dtype=np.complex128)
    for s in range(V):
        A11[3 * s:3 * s + 3, 3 * s:3 * s + 3] += m0 * np.eye(3)
    for t in range(dims[3]):
        for z in range(dims[2]):
            for y in range(dims[1]):
                for x in range(dims[0]):
                    c = [x, y, z, t]
                    s = site_index(c, dims)
                    for mu in range(4):
                        cp = list(c); cp[mu] = (cp[mu] + 1) % dims[mu]
                        cm = list(c); cm[mu] = (cm[mu] - 1) % dims[mu]
                        sp, sm = site_index(cp, dims), site_index(cm, dims)
                        # forward hop: row block x, column block x+mu, matrix U_mu(x) / W_mu(x)
                        A11[3 * s:3 * s + 3, 3 * sp:3 * sp + 3] += U[mu, s]
                        A12[3 * s:3 * s + 3, 3 * sp:3 * sp + 3] += kappa * W[mu, s]
                        # backward hop: column block y = x-mu, matrix U_mu(y)^H / -W_mu(y)^T
                        A11[3 * s:3 * s + 3, 3 * sm:3 * sm + 3] += U[mu, sm].conj().T
                        A12[3 * s:3 * s + 3, 3 * sm:3 * sm + 3] -= kappa * W[mu, sm].T
    return A11, A12


def dense_eigvals_brute(A: np.ndarray) -> np.ndarray:
    """All eigenvalues of a dense Hermitian matrix, ascending (LAPACK zheevd via numpy)."""
    return np.linalg.eigvalsh(A)
