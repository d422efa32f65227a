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


def constant_link_spectrum_batched(U0, W0, dims, m0, kappa):
    """The same spectrum as constant_link_spectrum, with H(p) built for all momenta at once and
    diagonalised as one batch of 6x6 Hermitian matrices (seconds even at 24^3 x 48)."""
    ks = np.meshgrid(*[2.0 * np.pi * np.arange(int(L)) / int(L) for L in dims], indexing="ij")
    P = np.stack([k.reshape(-1) for k in ks], axis=1)              # (V, 4)
    V = P.shape[0]
    H = np.zeros((V, 6, 6), dtype=np.complex128)
    idx = np.arange(3)
    H[:, idx, idx] = m0
    H[:, 3 + idx, 3 + idx] = m0
    for mu in range(4):
        e = np.exp(1j * P[:, mu])[:, None, None]
        a = U0[mu][None] * e + U0[mu].conj().T[None] / e
        c = U0[mu].conj()[None] * e + U0[mu].T[None] / e
        b = kappa * (W0[mu][None] * e - W0[mu].T[None] / e)
        H[:, :3, :3] += a
        H[:, 3:, 3:] += c
        H[:, :3, 3:] += b
        H[:, 3:, :3] += np.conj(np.transpose(b, (0, 2, 1)))
    return np.sort(np.linalg.eigvalsh(H).reshape(-1))


def distinct_pair_values(spec, count):
    """The lowest `count` eigenvalues once each, from a full spectrum in which every value appears
    twice (eq. (5)); returns (values, largest mismatch within a pair, smallest relative gap between
    consecutive values among the first count + 1)."""
    lo = spec[: 2 * (count + 1)].reshape(-1, 2)
    pair_mismatch = float(np.abs(lo[:, 0] - lo[:, 1]).max())
    vals = lo[:, 0]
    gap = float((np.diff(vals) / np.abs(vals[1:])).min())
    return vals[:count], pair_mismatch, gap
