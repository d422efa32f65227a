"""Pins for the Case A generator and the plain TRLAN of the oracle (Sec. 3: TRLAN is Algorithms 1-2
with W removed; Sec. 4, Case A: A = U diag(L, L) U^H with the constraints of eq. (5))."""
import numpy as np

from oracle import jsym
from oracle import trlan_jsym as tj
from paper_2001_07428_gb300 import inputs


def test_case_a_has_the_diagonal_block_form():
    n, h = 40, 20
    A11, A12, lam = inputs.case_a(n, 1)
    A = jsym.assemble_block_form(A11, A12)
    Jm = jsym.J_matrix(n)
    assert np.allclose(A, A.conj().T, atol=1e-14)
    assert np.allclose(Jm @ A @ Jm.T, A.T, atol=1e-14)                    # eq. (1)
    assert np.allclose(np.linalg.eigvalsh(A), np.sort(np.r_[lam, lam]), atol=1e-13)
    assert (lam > 0).all() and (lam < 1).all()


def test_plain_trlan_finds_each_eigenvalue_twice_at_about_twice_the_cost():
    A11, A12, lam = inputs.case_a(400, 3)
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    top = np.sort(lam)[::-1][:5]
    js = tj.trlan_jsym(mv, 400, 5, 50, 10, 1e-11, which="largest")
    tr = tj.trlan_jsym(mv, 400, 10, 100, 20, 1e-11, which="largest", use_w=False)   # parameters doubled
    assert np.abs(js["evals"] - top).max() < 1e-12
    assert np.abs(tr["evals"] - np.repeat(top, 2)).max() < 1e-12              # both members of each pair
    assert tr["n_matvec"] > 1.5 * js["n_matvec"]                             # the paper's N_MV claim
