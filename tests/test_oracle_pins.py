"""Pins for the CPU oracle: what the paper and the mathematics fix, independent of the oracle itself.

Each test names the passage it follows.  None of them compares the oracle with a
re-typed copy of its own formula: they use identities (Lemma 1, eq. (1)), brute-force
assembly from matrix entries, closed-form momentum-space spectra, textbook special
cases, and LAPACK on the assembled matrix.
"""
import numpy as np
import pytest

from oracle import jsym
from oracle import trlan_jsym as tj
from paper_2001_07428_gb300 import inputs
from tests import closed_form as cf


def _stencil_mv(U, W, dims, m0, kappa):
    return lambda x: jsym.stencil_matvec(U, W, dims, m0, kappa, x)


# ----------------------------------------------------------------------------- J (eq. (1), Sec. 1)
def test_canonical_J_is_skew_and_orthogonal():
    Jm = jsym.J_matrix(8)
    assert np.array_equal(Jm.T, -Jm)
    assert np.array_equal(Jm.T @ Jm, np.eye(8))
    x = inputs.random_vector(8, 3)
    assert np.allclose(jsym.apply_J(x), Jm @ x, atol=0)
    # J (J x*)* = J J x = -x
    assert np.allclose(jsym.pair(jsym.pair(x)), -x, atol=0)


@pytest.mark.parametrize("h", [1, 5, 50])
def test_dense_block_form_is_hermitian_J_symmetric(h):
    A11, A12 = inputs.dense_jsym(h, seed=h)
    A = jsym.assemble_block_form(A11, A12)
    Jm = jsym.J_matrix(2 * h)
    assert np.allclose(A, A.conj().T, atol=1e-14)
    assert np.allclose(Jm @ A @ Jm.T, A.T, atol=1e-13)   # J A J^{-1} = A^T, J^{-1} = J^T
    assert np.allclose(A12.T, -A12, atol=0)


# ----------------------------------------------------------------------------- Lemma 1 and Hermiticity
def _lemma1_and_hermitian(mv, n, scale):
    v = inputs.random_vector(n, 11)
    u = inputs.random_vector(n, 12)
    w = jsym.pair(v)
    Av = mv(v)
    tol = 1e-12 * scale * n
    assert abs(np.vdot(w, v)) < tol                      # w^H v = 0
    assert abs(np.vdot(w, Av)) < tol                     # w^H A v = 0
    assert abs(np.vdot(u, Av) - np.conj(np.vdot(v, mv(u)))) < tol
    # A (J v*) = J (A v)*  (J-symmetry with Hermiticity: J A^* = A J)
    assert np.allclose(mv(jsym.pair(v)), jsym.pair(Av), atol=tol)


def test_lemma1_dense():
    A11, A12 = inputs.dense_jsym(60, seed=4)
    _lemma1_and_hermitian(lambda x: jsym.dense_matvec(A11, A12, x), 120, 20.0)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 3, 4, 5), (8, 8, 8, 8)])
def test_lemma1_stencil(dims):
    U, W = inputs.stencil_links(dims, seed=2)
    n = 6 * inputs.lattice_volume(dims)
    _lemma1_and_hermitian(_stencil_mv(U, W, dims, 8.5, 0.3), n, 20.0)


# ----------------------------------------------------------------------------- stencil vs entry-wise assembly
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (3, 2, 4, 2), (2, 3, 3, 4)])
def test_stencil_matches_entrywise_assembly(dims):
    U, W = inputs.stencil_links(dims, seed=5)
    A11, A12 = jsym.stencil_blocks_dense(U, W, dims, 8.5, 0.3)
    assert np.allclose(A11, A11.conj().T, atol=1e-15)
    assert np.allclose(A12.T, -A12, atol=1e-15)
    A = jsym.assemble_block_form(A11, A12)
    n = A.shape[0]
    for seed in range(3):
        x = inputs.random_vector(n, 100 + seed)
        assert np.allclose(jsym.stencil_matvec(U, W, dims, 8.5, 0.3, x), A @ x, atol=1e-12)


def test_free_field_spectrum():
    dims = (3, 2, 4, 2)
    U, W = inputs.free_links(dims)
    A = jsym.assemble_block_form(*jsym.stencil_blocks_dense(U, W, dims, 8.5, 0.7))
    assert np.allclose(np.linalg.eigvalsh(A), cf.free_spectrum(dims, 8.5), atol=1e-12)


def test_constant_links_spectrum_brute_force():
    dims = (2, 3, 2, 3)
    U, W, U0, W0 = inputs.constant_links(dims, seed=7)
    A = jsym.assemble_block_form(*jsym.stencil_blocks_dense(U, W, dims, 8.5, 0.3))
    exact = cf.constant_link_spectrum(U0, W0, dims, 8.5, 0.3)
    assert np.allclose(np.linalg.eigvalsh(A), exact, atol=1e-11)


@pytest.mark.parametrize("dims", [(4, 6, 8, 4), (8, 8, 8, 8)])
def test_stencil_on_plane_waves(dims):
    """A(e^{ipx} phi) = e^{ipx} H(p) phi at any lattice size."""
    U, W, U0, W0 = inputs.constant_links(dims, seed=9)
    mv = _stencil_mv(U, W, dims, 8.5, 0.3)
    rng = np.random.default_rng(0)
    for _ in range(4):
        p = np.array([2 * np.pi * rng.integers(L) / L for L in dims])
        phi = inputs.complex_gaussian(rng, (6,))
        x = cf.plane_wave(dims, p, phi)
        expect = cf.plane_wave(dims, p, cf.H_of_p(U0, W0, 8.5, 0.3, p) @ phi)
        assert np.allclose(mv(x), expect, atol=1e-12)


# ----------------------------------------------------------------------------- Algorithm 1 against brute force
def _check_output_structure(out, mv, nev, tol):
    X = out["X"]
    Y = np.stack([jsym.pair(X[:, i]) for i in range(nev)], axis=1)
    assert np.allclose(X.conj().T @ X, np.eye(nev), atol=1e-12)     # X^H X = I
    assert np.abs(Y.conj().T @ X).max() < 1e-12                        # (J X*)^H X = O (eq. (5))
    for i in range(nev):
        r = mv(X[:, i]) - out["evals"][i] * X[:, i]
        assert np.linalg.norm(r) < tol
        # the partner is an eigenvector for the same eigenvalue (eq. (2))
        rp = mv(Y[:, i]) - out["evals"][i] * Y[:, i]
        assert np.linalg.norm(rp) < tol


def _check_mv_bounds(out, m, mwin, nev):
    """Eq. (30): m + (m-mwin-nev)(Nconv-1) <= N_MV <= m + (m-mwin)(Nconv-1)."""
    nc = out["n_restarts"]
    assert m + (m - mwin - nev) * (nc - 1) <= out["n_matvec"] <= m + (m - mwin) * (nc - 1)


def test_trlan_dense_n200_matches_brute_force():
    w = inputs.WORKLOADS["dense_n200"]
    A11, A12 = inputs.dense_jsym(w["n"] // 2, w["seed"])
    A = jsym.assemble_block_form(A11, A12)
    ev_all = np.linalg.eigvalsh(A)
    assert np.abs(ev_all[0::2] - ev_all[1::2]).max() < 1e-12          # every eigenvalue twice
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    out = tj.trlan_jsym(mv, w["n"], w["nev"], w["m"], w["mwin"], 1e-12)
    assert np.allclose(out["evals"], ev_all[0::2][: w["nev"]], rtol=1e-12, atol=1e-12)
    _check_output_structure(out, mv, w["nev"], 1e-12)
    _check_mv_bounds(out, w["m"], w["mwin"], w["nev"])


def test_trlan_largest_dense():
    A11, A12 = inputs.dense_jsym(80, 3)
    ev_all = np.linalg.eigvalsh(jsym.assemble_block_form(A11, A12))
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    out = tj.trlan_jsym(mv, 160, 6, 24, 12, 1e-11, which="largest")
    assert np.allclose(out["evals"], ev_all[::-1][0::2][:6], atol=1e-11)
    _check_output_structure(out, mv, 6, 1e-11)


def test_trlan_stencil_4x4x4x4_matches_brute_force():
    dims = (4, 4, 4, 4)
    U, W = inputs.stencil_links(dims, seed=1)
    A = jsym.assemble_block_form(*jsym.stencil_blocks_dense(U, W, dims, 8.5, 0.3))
    ev_all = np.linalg.eigvalsh(A)
    mv = _stencil_mv(U, W, dims, 8.5, 0.3)
    out = tj.trlan_jsym(mv, A.shape[0], 10, 40, 20, 1e-12)
    assert np.allclose(out["evals"], ev_all[0::2][:10], atol=1e-11)
    _check_output_structure(out, mv, 10, 1e-12)
    _check_mv_bounds(out, 40, 20, 10)


def test_trlan_A12_zero_reduces_to_A11():
    """A12 = 0: spectrum(A) = spectrum(A11), each value twice (a textbook Hermitian eigensolve)."""
    A11, _ = inputs.dense_jsym(90, 8)
    A12 = np.zeros_like(A11)
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    out = tj.trlan_jsym(mv, 180, 8, 30, 16, 1e-12)
    assert np.allclose(out["evals"], np.linalg.eigvalsh(A11)[:8], atol=1e-11)


def test_trlan_constant_links_closed_form():
    """Translation-invariant links at 6^4 (n = 7776): pinned to the momentum-space spectrum."""
    dims = (6, 6, 6, 6)
    U, W, U0, W0 = inputs.constant_links(dims, seed=21)
    exact = cf.constant_link_spectrum(U0, W0, dims, 8.5, 0.3)
    distinct = exact[0::2]
    nev = 6
    assert np.abs(exact[0::2] - exact[1::2])[: nev + 1].max() < 1e-10
    assert np.diff(distinct[: nev + 2]).min() > 1e-6    # no degeneracy beyond the J pair
    mv = _stencil_mv(U, W, dims, 8.5, 0.3)
    # v1 = (1,..,1) is the p = 0 plane wave, an invariant subspace here: start at random
    with pytest.raises(tj.BreakdownError):
        tj.trlan_jsym(mv, 6 * 6 ** 4, nev, 40, 12, 1e-11)
    v1 = inputs.random_vector(6 * 6 ** 4, 5)
    out = tj.trlan_jsym(mv, 6 * 6 ** 4, nev, 40, 12, 1e-11, v1=v1)
    assert np.allclose(out["evals"], distinct[:nev], atol=1e-10)


# ----------------------------------------------------------------------------- invariants during the iteration
def test_corollaries_and_krylov_schur_relation():
    """Cor. 1-2: V^H W = O and V^H A W = O; eq. (6) / Krylov-Schur form; V^H V = I."""
    A11, A12 = inputs.dense_jsym(100, 0)
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    A = jsym.assemble_block_form(A11, A12)
    seen = []

    def hook(V, T, k, m):
        Vm1 = V[:, : m + 1]
        Wm1 = np.stack([jsym.pair(Vm1[:, i]) for i in range(m + 1)], axis=1)
        assert np.allclose(Vm1.conj().T @ Vm1, np.eye(m + 1), atol=1e-12)
        assert np.abs(Vm1.conj().T @ Wm1).max() < 1e-12
        assert np.abs(Vm1.conj().T @ (A @ Wm1)).max() < 1e-10
        Vm = V[:, :m]
        R = A @ Vm - Vm @ T[:m, :m] - np.outer(V[:, m], T[m, :m])
        assert np.abs(R).max() < 1e-11
        seen.append(k)

    tj.trlan_jsym(mv, 200, 10, 30, 15, 1e-12, on_lanczos=hook)
    assert len(seen) > 2 and seen[0] == 0 and min(seen[1:]) >= 15


def test_invalid_parameters():
    mv = lambda x: x
    for args in [(7, 2, 5, 2), (200, 5, 5, 2), (200, 5, 100, 2), (200, 5, 20, -1)]:
        with pytest.raises(ValueError):
            tj.trlan_jsym(mv, *args, 1e-8)
