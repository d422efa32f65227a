"""Pins of the oracle's inertia count (oracle/inertia.py) and the completeness of the 8^4 golden.

* count_below against brute force (LAPACK eigvalsh) on random Hermitian matrices, at shifts between
  eigenvalues, including a zero-diagonal matrix whose factorisation needs 2x2 pivots;
* on a Hermitian J-symmetric matrix the count is even at every shift between eigenvalue pairs (eq. (2));
* the stored inertia of the 8^4 stencil (tests/golden/stencil_8x8x8x8_inertia.json, written by
  tests/golden/make_inertia.py with the oracle only) shows that the 20 eigenvalues of the 8^4 golden
  are the 20 smallest: 40 eigenvalues (20 doubly degenerate pairs) lie below a shift between
  lambda_20 and lambda_21.
"""
import json
import os

import numpy as np
import pytest

from oracle import inertia, jsym
from paper_2001_07428_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _hermitian(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return (X + X.conj().T) / 2


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (50, 3), (151, 4)])
def test_count_below_matches_brute_force(n, seed):
    A = _hermitian(n, seed)
    lam = np.linalg.eigvalsh(A)
    shifts = list((lam[:-1] + lam[1:]) / 2) + [lam[0] - 1.0, lam[-1] + 1.0]
    for sigma in shifts[:: max(1, len(shifts) // 12)]:
        assert inertia.count_below(A, sigma) == int((lam < sigma).sum())


def test_count_below_with_two_by_two_pivots():
    """A zero diagonal forces Bunch-Kaufman 2x2 pivots; counting only D's diagonal would be wrong."""
    A = _hermitian(60, 9)
    A[np.diag_indices_from(A)] = 0.0
    lam = np.linalg.eigvalsh(A)
    for sigma in (0.0, (lam[10] + lam[11]) / 2, (lam[40] + lam[41]) / 2):
        assert inertia.count_below(A, sigma) == int((lam < sigma).sum())


def test_a_count_of_the_diagonal_alone_is_caught(monkeypatch):
    """Planted mistake: ignoring the 2x2 blocks of D (counting only its diagonal) must fail the pin."""
    import scipy.linalg

    A = _hermitian(60, 9)
    A[np.diag_indices_from(A)] = 0.0
    lam = np.linalg.eigvalsh(A)
    real_ldl = scipy.linalg.ldl

    def diagonal_only(*a, **k):
        lu, d, perm = real_ldl(*a, **k)
        return lu, np.diag(np.diag(d)), perm

    monkeypatch.setattr(inertia.scipy.linalg, "ldl", diagonal_only)
    assert any(inertia.count_below(A, s) != int((lam < s).sum()) for s in (0.0, (lam[10] + lam[11]) / 2))


def test_count_is_even_for_a_jsymmetric_matrix():
    A11, A12 = inputs.dense_jsym(40, 3)
    A = jsym.assemble_block_form(A11, A12)
    lam = np.linalg.eigvalsh(A)
    for i in range(1, 40, 7):                          # between the pairs (2i - 1, 2i)
        sigma = (lam[2 * i - 1] + lam[2 * i]) / 2
        c = inertia.count_below(A, sigma)
        assert c == 2 * i and c % 2 == 0


def test_count_on_a_small_stencil_matches_brute_force():
    dims = (3, 2, 2, 2)
    U, W = inputs.stencil_links(dims, 4)
    A = jsym.assemble_block_form(*jsym.stencil_blocks_dense(U, W, dims, 8.5, 0.3))
    lam = np.linalg.eigvalsh(A)
    for i in (2, 10, 30):
        sigma = (lam[i - 1] + lam[i]) / 2
        assert inertia.count_below(A, sigma) == i


def test_the_8x8x8x8_golden_is_complete():
    rec = json.load(open(os.path.join(GOLDEN, "stencil_8x8x8x8_inertia.json")))
    gold = json.load(open(os.path.join(GOLDEN, "stencil_8x8x8x8.json")))
    nev = len(gold["evals"])
    assert rec["nev"] == nev and rec["workload"] == gold["workload"]
    lam_nev, lam_next = max(gold["evals"]), rec["lambda_next"]
    assert lam_nev < rec["sigma"] < lam_next              # the shift lies in the gap above lambda_nev
    assert rec["count_below"] == 2 * nev                  # every eigenvalue below it was found (each twice)
