"""Closed-form spectra used to pin the oracle (test-side, independent of oracle/ and the library).

Translation-invariant links (U_mu, W_mu the same at every site) make the stencil
operator diagonal in momentum space: on psi(x) = exp(i p.x) phi with p_mu = 2 pi k_mu / L_mu,
A acts as the 6x6 Hermitian matrix

    H(p) = [[a(p), b(p)], [b(p)^H, c(p)]]
    a(p) = m0 + sum_mu (U_mu e^{i p_mu} + U_mu^H e^{-i p_mu})
    c(p) = m0 + sum_mu (U_mu^* e^{i p_mu} + U_mu^T e^{-i p_mu})
    b(p) = kappa sum_mu (W_mu e^{i p_mu} - W_mu^T e^{-i p_mu})

(derived by inserting the plane wave into the two block rows of eq. (4)).  With
U = I and W = 0 every eigenvalue is m0 + 2 sum_mu cos(p_mu).
"""
from __future__ import annotations

import itertools

import numpy as np


def momenta(dims):
    for ks in itertools.product(*[range(int(L)) for L in dims]):
        yield np.array([2.0 * np.pi * k / L for k, L in zip(ks, dims)])


def H_of_p(U0, W0, m0, kappa, p):
    a = m0 * np.eye(3, dtype=np.complex128)
    c = m0 * np.eye(3, dtype=np.complex128)
    b = np.zeros((3, 3), dtype=np.complex128)
    for mu in range(4):
        e = np.exp(1j * p[mu])
        a += U0[mu] * e + U0[mu].conj().T / e
        c += U0[mu].conj() * e + U0[mu].T / e
        b += kappa * (W0[mu] * e - W0[mu].T / e)
    return np.block([[a, b], [b.conj().T, c]])


def constant_link_spectrum(U0, W0, dims, m0, kappa):
    """All n = 6V eigenvalues, ascending."""
    vals = [np.linalg.eigvalsh(H_of_p(U0, W0, m0, kappa, p)) for p in momenta(dims)]
    return np.sort(np.concatenate(vals))


def plane_wave(dims, p, phi6):
    """The vector exp(i p.x) [phi1; phi2] in the canonical layout (x fastest)."""
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(range(Lt), range(Lz), range(Ly), range(Lx), indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t)).reshape(-1)
    x1 = (ph[:, None] * phi6[None, :3]).reshape(-1)
    x2 = (ph[:, None] * phi6[None, 3:]).reshape(-1)
    return np.concatenate([x1, x2])


def free_spectrum(dims, m0):
    vals = [m0 + 2.0 * np.sum(np.cos(p)) for p in momenta(dims)]
    return np.sort(np.repeat(vals, 6))
