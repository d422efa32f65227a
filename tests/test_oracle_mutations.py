"""Planted mistakes in the oracle (on the CPU) must be caught by the pins.

Each test plants one plausible error -- a wrong sign, a wrong link, a dropped
reorthogonalisation, a transposed eigenvector matrix -- and checks that the
corresponding pin fails.  This shows the pins are strong enough to trust the oracle.
"""
import numpy as np
import pytest

from oracle import jsym
from oracle import trlan_jsym as tj
from paper_2001_07428_gb300 import inputs


def _lemma1_residual(mv, n):
    v = inputs.random_vector(n, 11)
    return abs(np.vdot(jsym.pair(v), mv(v)))


def _hermiticity_residual(mv, n):
    u = inputs.random_vector(n, 12)
    v = inputs.random_vector(n, 13)
    return abs(np.vdot(u, mv(v)) - np.conj(np.vdot(v, mv(u))))


def test_wrong_sign_of_A12H_block_breaks_hermiticity():
    """Lemma 1 alone cannot see this sign (w^H A v stays 0); the Hermiticity pin does."""
    dims = (4, 4, 4, 4)
    U, W = inputs.stencil_links(dims, 2)
    n = 6 * 256

    def bad(x):
        h = n // 2
        y = jsym.stencil_matvec(U, W, dims, 8.5, 0.3, x)
        A12H_x1 = -np.conj(jsym.stencil_A12(W, dims, 0.3, np.conj(x[:h])))
        y[h:] -= 2 * A12H_x1                             # planted: +A12^* x1 instead of -A12^* x1
        return y

    good = lambda x: jsym.stencil_matvec(U, W, dims, 8.5, 0.3, x)
    assert _lemma1_residual(good, n) < 1e-9 and _hermiticity_residual(good, n) < 1e-9
    assert _hermiticity_residual(bad, n) > 1e-3


def test_untransposed_A22_breaks_lemma1():
    """A22 = A11 instead of A11^T keeps A Hermitian but breaks J-symmetry: Lemma 1 fails."""
    A11, A12 = inputs.dense_jsym(40, 1)
    bad = lambda x: np.concatenate([A11 @ x[:40] + A12 @ x[40:],
                                    A12.conj().T @ x[:40] + A11 @ x[40:]])
    assert _hermiticity_residual(bad, 80) < 1e-10
    good = lambda x: jsym.dense_matvec(A11, A12, x)
    assert _lemma1_residual(good, 80) < 1e-10
    assert _lemma1_residual(bad, 80) > 1e-3


def test_wrong_backward_link_breaks_entrywise_assembly():
    dims = (2, 3, 4, 2)
    U, W = inputs.stencil_links(dims, 5)
    A = jsym.assemble_block_form(*jsym.stencil_blocks_dense(U, W, dims, 8.5, 0.3))
    n = A.shape[0]
    x = inputs.random_vector(n, 1)
    orig = jsym._bwd

    def bad_bwd(f, mu):                                  # planted: backward shift along the wrong axis
        return orig(f, (mu + 1) % 4)

    try:
        jsym._bwd = bad_bwd
        y = jsym.stencil_matvec(U, W, dims, 8.5, 0.3, x)
    finally:
        jsym._bwd = orig
    assert not np.allclose(y, A @ x, atol=1e-8)


def _dense_case():
    A11, A12 = inputs.dense_jsym(100, 0)
    A = jsym.assemble_block_form(A11, A12)
    return A11, A12, np.linalg.eigvalsh(A)


def _passes_brute_force(out, ev_all, nev):
    X = out["X"]
    Y = np.stack([jsym.pair(X[:, i]) for i in range(nev)], axis=1)
    return (np.allclose(out["evals"], ev_all[0::2][:nev], atol=1e-10)
            and np.abs(Y.conj().T @ X).max() < 1e-10)


def test_dropping_W_reorthogonalisation_is_caught(monkeypatch):
    A11, A12, ev_all = _dense_case()
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    monkeypatch.setattr(tj, "pair", lambda x: np.zeros_like(x))   # planted: GS against W removed
    try:
        out = tj.trlan_jsym(mv, 200, 10, 30, 15, 1e-12, max_restarts=200)
    except (tj.NoConvergenceError, tj.BreakdownError):
        return
    assert not _passes_brute_force(out, ev_all, 10)


def test_transposed_ritz_vectors_are_caught(monkeypatch):
    A11, A12, ev_all = _dense_case()
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    real_eigh = tj.jacobi_eigh

    def transposed(Tm):
        lam, Z = real_eigh(Tm)
        return lam, Z.T.copy()                           # planted: Z transposed

    monkeypatch.setattr(tj, "jacobi_eigh", transposed)
    try:
        out = tj.trlan_jsym(mv, 200, 10, 30, 15, 1e-12, max_restarts=60)
    except (tj.NoConvergenceError, tj.BreakdownError):
        return
    assert not _passes_brute_force(out, ev_all, 10)


def test_normalising_by_b0_breaks_orthonormality(monkeypatch):
    """Reading R1: Algorithm 2 taken literally divides by the pre-pass norm."""
    A11, A12, _ = _dense_case()
    A = jsym.assemble_block_form(A11, A12)
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    n, m = 200, 20
    V = np.zeros((n, m + 1), dtype=np.complex128)
    T = np.zeros((m + 1, m + 1))
    V[:, 0] = 1 / np.sqrt(n)
    real_norm = np.linalg.norm
    calls = {"k": 0}

    def norm_b0(y):
        # planted: report the norm as if the last pass had not happened (b0 instead of b1)
        calls["k"] += 1
        return real_norm(y) * (1.3 if calls["k"] % 2 == 0 else 1.0)

    monkeypatch.setattr(tj.np.linalg, "norm", norm_b0)
    tj.lanczos_jsym(mv, V, T, 0, m)
    monkeypatch.undo()
    G = V.conj().T @ V
    assert not np.allclose(G, np.eye(m + 1), atol=1e-8)
