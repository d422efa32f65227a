"""Pins for the invert-mode oracle (Algorithm 1's invert mode with CG as the inner solver, Sec. 4):
CG against a direct solve, CG's finite termination on an operator with few distinct eigenvalues and
the monotone A-norm error (textbook properties), and invert-mode J-TRLan against brute-force
diagonalisation, with its residual estimate c |t_{m+1,i} ev(i)| checked against the true residual."""
import numpy as np
import pytest

from oracle import jsym
from oracle import trlan_jsym as tj
from oracle.cg import NotPositiveDefiniteError, cg
from paper_2001_07428_gb300 import inputs


def _hpd(n, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return G @ G.conj().T / n + np.eye(n)


def test_cg_matches_direct_solve():
    M = _hpd(40, 1)
    b = inputs.random_vector(40, 2)
    x, its = cg(lambda v: M @ v, b, rtol=1e-14)
    ref = np.linalg.solve(M, b)
    assert np.linalg.norm(x - ref) < 1e-11 * np.linalg.norm(ref)
    assert 0 < its <= 200


def test_cg_terminates_after_as_many_steps_as_distinct_eigenvalues():
    # exact arithmetic: CG ends after k steps when b meets k distinct eigenvalues
    d = np.repeat([1.0, 2.0, 3.5, 7.0, 11.0], 6)
    b = inputs.random_vector(30, 3)
    x, its = cg(lambda v: d * v, b, rtol=1e-10)
    assert its <= 5
    assert np.linalg.norm(d * x - b) <= 1e-10 * np.linalg.norm(b)


def test_cg_a_norm_error_never_grows():
    M = _hpd(50, 4)
    b = inputs.random_vector(50, 5)
    hist = []
    cg(lambda v: M @ v, b, rtol=1e-13, history=hist)
    xs = np.linalg.solve(M, b)
    e = [np.sqrt(np.vdot(x - xs, M @ (x - xs)).real) for x in hist]
    assert all(e[i + 1] <= e[i] * (1 + 1e-12) + 1e-14 for i in range(len(e) - 1))
    assert e[-1] < 1e-10 * e[0]


def test_cg_rejects_an_indefinite_operator():
    d = np.array([1.0, -2.0, 3.0, 4.0])
    with pytest.raises(NotPositiveDefiniteError):
        cg(lambda v: d * v, np.ones(4, dtype=complex))


def _pd_jsym(h, seed):
    """A Hermitian J-symmetric matrix shifted to lambda_min = 1 (A11 + s I keeps eq. (1))."""
    A11, A12 = inputs.dense_jsym(h, seed)
    lam = np.linalg.eigvalsh(jsym.assemble_block_form(A11, A12))
    A11 = A11 + (1.0 - lam[0]) * np.eye(h)
    A = jsym.assemble_block_form(A11, A12)
    return A11, A12, A


def test_invert_mode_matches_brute_force():
    A11, A12, A = _pd_jsym(60, 7)
    n = 120
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    out = tj.trlan_jsym(mv, n, 5, 20, 10, 1e-10, solve=lambda b: np.linalg.solve(A, b))
    lam = np.linalg.eigvalsh(A)
    assert np.allclose(lam[0::2], lam[1::2], atol=1e-9 * lam[-1])      # every eigenvalue twice (eq. (5))
    bf = lam[0::2][:5]
    assert np.abs(out["evals"] - bf).max() < 1e-10 * np.abs(bf).max()
    X = out["X"]
    for i in range(5):
        assert np.linalg.norm(mv(X[:, i]) - out["evals"][i] * X[:, i]) < 1e-10
    assert np.abs(X.conj().T @ X - np.eye(5)).max() < 1e-10


def test_invert_mode_residual_estimate_equals_the_true_residual():
    # with exact solves, c |t_{m+1,i}| / lambda_i is the residual of A at the Ritz pair (R20)
    A11, A12, A = _pd_jsym(60, 8)
    n = 120
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    out = tj.trlan_jsym(mv, n, 6, 20, 8, 1e-6, solve=lambda b: np.linalg.solve(A, b))
    last = out["history"][-1]
    assert last["icnv"] == 6
    # pairs locked at an earlier restart are decoupled (t_{m+1,i} = 0, estimate 0); the ones that
    # converged at the last restart carry the estimate of this restart
    fresh = [i for i in range(6) if last["res_est"][i] > 0]
    assert fresh
    ev_by_value = {round(e, 12): r for e, r in zip(out["evals"], out["res"])}
    for i in fresh:
        r = ev_by_value[round(last["ev"][i], 12)]
        assert abs(last["res_est"][i] - r) <= 1e-3 * r + 1e-13


def test_invert_mode_with_cg_and_plain_trlan():
    # the inner solver is the oracle's CG; plain TRLAN (W removed) in invert mode finds the same
    # smallest eigenvalues, and both count A^{-1} applications as N_MV
    A11, A12, A = _pd_jsym(50, 9)
    n = 100
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    solve = lambda b: cg(mv, b, rtol=1e-13)[0]
    js = tj.trlan_jsym(mv, n, 4, 16, 8, 1e-9, solve=solve)
    tr = tj.trlan_jsym(mv, n, 8, 32, 16, 1e-9, solve=solve, use_w=False)
    lam = np.linalg.eigvalsh(A)
    assert np.abs(js["evals"] - lam[0::2][:4]).max() < 1e-9
    assert np.abs(tr["evals"] - lam[:8]).max() < 1e-9
    assert js["n_matvec"] > 0 and tr["n_matvec"] > 0
