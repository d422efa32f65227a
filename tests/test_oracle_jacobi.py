"""Pins for the oracle's cyclic Jacobi eigensolver (the T_m = Z Lambda Z^T of Algorithm 1).

Closed forms (diagonal, 2 x 2, the tridiagonal Toeplitz matrix), the defining identities
(Z^T Z = I, Z Lambda Z^T = T), a library routine (LAPACK through numpy.linalg.eigvalsh) on
random and on arrowhead-plus-tridiagonal matrices shaped like T-bar after a thick restart,
and a planted mistake that the reconstruction pin catches.
"""
import numpy as np
import pytest

from oracle import jacobi
from oracle.jacobi import jacobi_eigh


def _check(T, lam, Z, tol=1e-13):
    m = T.shape[0]
    scale = max(np.abs(T).max(), 1.0)
    assert np.all(np.diff(lam) >= 0)
    assert np.abs(Z.T @ Z - np.eye(m)).max() < tol * m
    assert np.abs(Z @ np.diag(lam) @ Z.T - T).max() < tol * m * scale


def test_diagonal_and_two_by_two_closed_forms():
    lam, Z = jacobi_eigh(np.diag([3.0, -1.0, 2.0]))
    assert np.array_equal(lam, [-1.0, 2.0, 3.0])
    a, b, c = 2.0, 0.75, -1.0                      # eigenvalues (a+c)/2 -+ sqrt(((a-c)/2)^2 + b^2)
    T = np.array([[a, b], [b, c]])
    lam, Z = jacobi_eigh(T)
    r = np.hypot((a - c) / 2, b)
    assert np.allclose(lam, [(a + c) / 2 - r, (a + c) / 2 + r], rtol=0, atol=1e-15)
    _check(T, lam, Z)


@pytest.mark.parametrize("m", [3, 17, 60])
def test_tridiagonal_toeplitz_closed_form(m):
    a, b = 1.5, -0.4                               # eigenvalues a + 2 b cos(k pi / (m + 1))
    T = np.diag(np.full(m, a)) + np.diag(np.full(m - 1, b), 1) + np.diag(np.full(m - 1, b), -1)
    lam, Z = jacobi_eigh(T)
    ref = np.sort(a + 2 * b * np.cos(np.arange(1, m + 1) * np.pi / (m + 1)))
    assert np.abs(lam - ref).max() < 1e-14 * m
    _check(T, lam, Z)


@pytest.mark.parametrize("m,seed", [(8, 0), (40, 1), (120, 2)])
def test_random_symmetric_against_lapack(m, seed):
    A = np.random.default_rng(seed).standard_normal((m, m))
    T = A + A.T
    lam, Z = jacobi_eigh(T)
    assert np.abs(lam - np.linalg.eigvalsh(T)).max() < 1e-14 * m * np.abs(T).max()
    _check(T, lam, Z)


def test_thick_restart_shape_against_lapack():
    """diag(lambda_1..k), the arrow row k+1 (some couplings at rounding level, as locked pairs
    leave them), then a tridiagonal tail: the T-bar of Algorithm 1 after a restart."""
    rng = np.random.default_rng(3)
    m, k = 60, 25
    T = np.zeros((m, m))
    T[np.arange(k), np.arange(k)] = np.sort(rng.uniform(1.0, 2.0, k))
    arrow = rng.standard_normal(k) * np.where(np.arange(k) < 5, 1e-17, 1e-3)
    T[k, :k] = T[:k, k] = arrow
    T[np.arange(k, m), np.arange(k, m)] = rng.uniform(1.0, 18.0, m - k)
    off = rng.uniform(0.5, 3.0, m - k - 1)
    T[np.arange(k + 1, m), np.arange(k, m - 1)] = off
    T[np.arange(k, m - 1), np.arange(k + 1, m)] = off
    lam, Z = jacobi_eigh(T)
    assert np.abs(lam - np.linalg.eigvalsh(T)).max() < 1e-13 * np.abs(T).max()
    _check(T, lam, Z)


def test_planted_wrong_rotation_sign_is_caught(monkeypatch):
    """Rotating Z with the transposed rotation leaves the eigenvalues (read off the diagonal of A)
    right but breaks the reconstruction Z Lambda Z^T = T."""
    T = np.random.default_rng(4).standard_normal((12, 12))
    T = T + T.T
    src = open(jacobi.__file__).read()
    bad_src = src.replace("Z[:, p] = c * zp - s * zq", "Z[:, p] = c * zp + s * zq").replace(
        "Z[:, q] = s * zp + c * zq", "Z[:, q] = -s * zp + c * zq")
    assert bad_src != src
    ns = {}
    exec(compile(bad_src, "jacobi_planted", "exec"), ns)
    lam, Z = ns["jacobi_eigh"](T)
    assert np.abs(lam - np.linalg.eigvalsh(T)).max() < 1e-12
    assert np.abs(Z @ np.diag(lam) @ Z.T - T).max() > 1e-3


def test_negligible_couplings_do_not_overflow():
    """A coupling 1e-300 next to a diagonal gap of 1 makes tau^2 overflow in the textbook formula; the
    rotation then tends to the identity (t -> 1/(2 tau)), and the result is the diagonal."""
    import warnings
    T = np.array([[1.0, 1e-300, 0.0], [1e-300, 2.0, 0.3], [0.0, 0.3, 5.0]])
    with warnings.catch_warnings():
        warnings.simplefilter("error")
        lam, Z = jacobi_eigh(T)
    assert np.abs(lam - np.linalg.eigvalsh(T)).max() < 1e-14
    _check(T, lam, Z)
