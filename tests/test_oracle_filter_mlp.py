"""Pins for the filter and MLP oracles: independent routes to the same numbers (eigendecomposition
instead of the three-term recurrence, quadrature instead of the closed-form coefficients, finite
differences instead of back-propagation, the first Adam step in closed form), invariants (J-symmetry
of p(A), positivity and -- up to the kernel's 1e-5 ripple -- monotonicity of the Jackson-damped
step) and special cases."""
import numpy as np
import pytest

from oracle import filter as flt
from oracle import jsym
from oracle import mlp
from paper_2001_07428_gb300 import inputs


def _dense(h, seed):
    A11, A12 = inputs.dense_jsym(h, seed)
    return A11, A12, jsym.assemble_block_form(A11, A12)


# ----------------------------------------------------------------------------- p(A)
def test_apply_poly_matches_the_eigendecomposition_route():
    A11, A12, A = _dense(12, 3)
    lam, U = np.linalg.eigh(A)
    a, b = lam[0] - 0.3, lam[-1] + 0.2
    rng = np.random.default_rng(0)
    coeffs = rng.standard_normal(13)
    x = inputs.random_vector(24, 5)
    got = flt.apply_poly(lambda v: jsym.dense_matvec(A11, A12, v), x, coeffs, a, b)
    c, e = flt.window(a, b)
    ref = U @ (flt.eval_poly(coeffs, (lam - c) / e) * (U.conj().T @ x))   # T_k(cos t) = cos(k t)
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


def test_filtered_operator_is_hermitian_J_symmetric():
    A11, A12, A = _dense(6, 9)
    lam = np.linalg.eigvalsh(A)
    coeffs = flt.damped_step_coeffs(-0.2, 16)
    n = 12
    P = np.stack([flt.apply_poly(lambda v: jsym.dense_matvec(A11, A12, v), np.eye(n)[:, i].astype(complex),
                                 coeffs, lam[0] - 1, lam[-1] + 1) for i in range(n)], axis=1)
    Jm = jsym.J_matrix(n)
    assert np.allclose(P, P.conj().T, atol=1e-12)
    assert np.allclose(Jm @ P @ Jm.T, P.T, atol=1e-12)      # eq. (1) for B = p(A)
    x = inputs.random_vector(n, 2)
    assert abs(np.vdot(jsym.pair(x), P @ x)) < 1e-12 * np.linalg.norm(P @ x) * np.linalg.norm(x)   # Lemma 1


# ----------------------------------------------------------------------------- coefficients
@pytest.mark.parametrize("tau", [-0.7, 0.0, 0.35])
def test_step_coefficients_match_chebyshev_gauss_quadrature(tau):
    M = 400000
    t = np.pi * (np.arange(M) + 0.5) / M
    f = (np.cos(t) <= tau).astype(float)
    k = np.arange(21)
    quad = 2.0 / M * (np.cos(np.outer(k, t)) @ f)
    quad[0] *= 0.5
    assert np.abs(flt.step_coeffs(tau, 20) - quad).max() < 1e-4


def test_step_special_cases():
    assert np.allclose(flt.step_coeffs(1.0, 10), np.r_[1.0, np.zeros(10)], atol=1e-15)    # f = 1
    assert np.allclose(flt.step_coeffs(-1.0, 10), np.zeros(11), atol=1e-15)               # f = 0


def test_jackson_damped_step_is_in_unit_interval_and_monotone():
    j = flt.jackson(64)
    assert abs(j[0] - 1.0) < 1e-15 and (np.abs(j) <= 1.0 + 1e-15).all()
    x = np.linspace(-1, 1, 20001)
    for tau in (-0.9, -0.3, 0.4):
        p = flt.eval_poly(flt.damped_step_coeffs(tau, 64), x)
        assert p.min() > -1e-12 and p.max() < 1 + 1e-12       # a non-negative kernel keeps [0, 1]
        assert (np.diff(p) <= 1e-5).all()                    # non-increasing up to the kernel's ripple
        assert p[x >= tau + 0.25].max() < 0.01
        if tau - 0.25 > -1:
            assert p[x <= tau - 0.25].min() > 0.99


def test_filter_ranks_the_wanted_eigenvalues_first():
    A11, A12, A = _dense(30, 4)
    lam = np.linalg.eigvalsh(A)[0::2]                      # one of each J pair
    a, b = lam[0] - 0.5, lam[-1] + 0.5
    tau = flt.cut_to_tau(0.5 * (lam[4] + lam[5]), a, b)
    c, e = flt.window(a, b)
    p = flt.eval_poly(flt.damped_step_coeffs(tau, 64), (lam - c) / e)
    assert p[:5].min() > p[5:].max()


# ----------------------------------------------------------------------------- MLP
F, H, O = 3, 5, 4


def _theta(seed):
    return np.random.default_rng(seed).standard_normal(mlp.n_params(F, H, O)) * 0.7


def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    X, T = rng.standard_normal((7, F)), rng.standard_normal((7, O))
    th = _theta(2)
    _, g = mlp.gradient(th, X, T, F, H, O)
    fd = np.empty_like(th)
    h = 1e-6
    for i in range(th.size):
        e = np.zeros_like(th)
        e[i] = h
        fd[i] = (mlp.loss(th + e, X, T, F, H, O) - mlp.loss(th - e, X, T, F, H, O)) / (2 * h)
    assert np.abs(g - fd).max() < 1e-7 * max(1.0, np.abs(fd).max())


def test_mlp_constant_output_case():
    # W3 = 0: Y = b3 for every sample, so dL/db3 = 2 (b3 - mean(T)) / O and the hidden layers get no gradient
    rng = np.random.default_rng(3)
    X, T = rng.standard_normal((6, F)), rng.standard_normal((6, O))
    th = _theta(4)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(th, F, H, O)
    W3[:] = 0.0
    L, g = mlp.gradient(th, X, T, F, H, O)
    assert abs(L - np.mean((b3 - T) ** 2)) < 1e-14
    gW1, gb1, gW2, gb2, gW3, gb3 = mlp.unpack(g, F, H, O)
    assert np.allclose(gb3, 2.0 * (b3 - T.mean(axis=0)) / O, atol=1e-14)
    for z in (gW1, gb1, gW2, gb2):
        assert np.abs(z).max() == 0.0


def test_mlp_forward_by_hand():
    # F = H = O = 1: Y = w3 tanh(w2 tanh(w1 x + b1) + b2) + b3
    th = np.array([0.5, -0.1, 2.0, 0.3, -1.5, 0.25])
    x = 0.8
    ref = -1.5 * np.tanh(2.0 * np.tanh(0.5 * x - 0.1) + 0.3) + 0.25
    Y, _, _ = mlp.forward(th, np.array([[x]]), 1, 1, 1)
    assert abs(Y[0, 0] - ref) < 1e-15


def test_adam_first_step_moves_each_parameter_by_lr():
    g = np.array([3.0, -2e-3, 0.5])
    th, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(th, -0.01 * np.sign(g), atol=1e-15)    # m_hat / sqrt(v_hat) = g / |g| at t = 1
