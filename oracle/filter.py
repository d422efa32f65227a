"""Polynomial spectral filters p(A) with real coefficients (oracle, test-only).

The paper runs J-TRLan on A itself; it has no filter.  The filtered form runs the same method
on B = p(A).  Because p has real coefficients and A is Hermitian J-symmetric, B is Hermitian and
J B J^{-1} = p(J A J^{-1}) = p(A^T) = p(A)^T, so B is Hermitian J-symmetric too (eq. (1)) and
Algorithm 1 applies to it unchanged; its eigenvectors are those of A, with eigenvalues p(lambda).

Definitions used here (standard, e.g. Rivlin, "Chebyshev Polynomials"):

* window [a, b] containing the spectrum; c = (a + b)/2, e = (b - a)/2; A_hat = (A - c I)/e.
* Chebyshev polynomials T_0 = 1, T_1(x) = x, T_{k+1} = 2 x T_k - T_{k-1}; T_k(cos t) = cos(k t).
* p(A) = sum_{k=0}^{d} g_k T_k(A_hat).
* step filter: f(x) = 1 for x <= tau, 0 for x > tau (x in [-1, 1]).  Its Chebyshev coefficients
  are c_0 = (pi - arccos tau)/pi and c_k = -2 sin(k arccos tau)/(pi k) (k >= 1), from
  c_k = (2/pi) int_0^pi f(cos t) cos(k t) dt.
* Jackson damping (kernel polynomial method, Weisse, Wellein, Alvermann and Fehske, Rev. Mod.
  Phys. 78, 275 (2006)) with N = d + 1 moments:
  j_k = [(N - k + 1) cos(pi k/(N+1)) + sin(pi k/(N+1)) cot(pi/(N+1))] / (N + 1).
  The damped expansion is the convolution (in the angle t) of f with a non-negative kernel, so it
  stays in [0, 1]; it is non-increasing up to ripples of order 1e-5 at degree 64.
"""
from __future__ import annotations

import numpy as np


def window(a: float, b: float):
    """(c, e) of the affine map x = (lambda - c)/e taking [a, b] onto [-1, 1]."""
    return 0.5 * (a + b), 0.5 * (b - a)


def apply_poly(matvec, x: np.ndarray, coeffs, a: float, b: float) -> np.ndarray:
    """p(A) x = sum_k coeffs[k] T_k(A_hat) x by the three-term recurrence, in FP64."""
    c, e = window(a, b)
    t_prev = np.asarray(x, dtype=np.complex128)
    acc = coeffs[0] * t_prev
    if len(coeffs) == 1:
        return acc
    t_cur = (matvec(t_prev) - c * t_prev) / e
    acc = acc + coeffs[1] * t_cur
    for k in range(2, len(coeffs)):
        t_next = 2.0 * (matvec(t_cur) - c * t_cur) / e - t_prev
        acc = acc + coeffs[k] * t_next
        t_prev, t_cur = t_cur, t_next
    return acc


def eval_poly(coeffs, x: np.ndarray) -> np.ndarray:
    """p(x) = sum_k coeffs[k] T_k(x) for real x in [-1, 1], through T_k(cos t) = cos(k t)."""
    t = np.arccos(np.clip(x, -1.0, 1.0))
    k = np.arange(len(coeffs))
    return np.cos(np.outer(t, k)) @ np.asarray(coeffs, dtype=np.float64)


def step_coeffs(tau: float, degree: int) -> np.ndarray:
    """Undamped Chebyshev coefficients c_0..c_degree of the step f(x) = [x <= tau]."""
    th = np.arccos(np.clip(tau, -1.0, 1.0))
    c = np.empty(degree + 1)
    c[0] = (np.pi - th) / np.pi
    k = np.arange(1, degree + 1)
    c[1:] = -2.0 * np.sin(k * th) / (np.pi * k)
    return c


def jackson(degree: int) -> np.ndarray:
    """Jackson damping factors j_0..j_degree for N = degree + 1 moments."""
    N = degree + 1
    k = np.arange(degree + 1)
    q = np.pi / (N + 1)
    return ((N - k + 1) * np.cos(q * k) + np.sin(q * k) / np.tan(q)) / (N + 1)


def damped_step_coeffs(tau: float, degree: int) -> np.ndarray:
    """g_k = j_k c_k: the Jackson-damped step filter used as the training target."""
    return jackson(degree) * step_coeffs(tau, degree)


def cut_to_tau(cut: float, a: float, b: float) -> float:
    """The window coordinate of an eigenvalue cut."""
    c, e = window(a, b)
    return (cut - c) / e
