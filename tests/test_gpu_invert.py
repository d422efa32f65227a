"""GPU parity of Algorithm 1's invert mode (the Lanczos product A^{-1} v_j by CG, Sec. 4) through
the C ABI, against brute-force diagonalisation, the invert-mode oracle and the normal-mode solve.

Tolerances: eigenvalues within 1e-10 relative of brute force / the oracle; true residuals
||A x - lambda x|| with unit x below the solve tolerance, recomputed here with the oracle's matvec.
"""
import numpy as np
import pytest

from oracle import jsym
from oracle import trlan_jsym as tj
from paper_2001_07428_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2001_07428_gb300 import binding
    binding.load()


def _pd_jsym(h, seed):
    A11, A12 = inputs.dense_jsym(h, seed)
    lam = np.linalg.eigvalsh(jsym.assemble_block_form(A11, A12))
    A11 = A11 + (1.0 - lam[0]) * np.eye(h)    # lambda_min = 1; A11 + s I keeps eq. (1)
    return A11, A12, jsym.assemble_block_form(A11, A12)


def _solver(**kw):
    from paper_2001_07428_gb300.solver import JTRLan
    return JTRLan(device="cuda:0", **kw)


def _check(ev, X, mv, tol, ref):
    Xh = X.cpu().numpy()
    assert np.abs(ev - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.abs(Xh.conj().T @ Xh - np.eye(len(ev))).max() < 1e-10
    for i in range(len(ev)):
        assert np.linalg.norm(mv(Xh[:, i]) - ev[i] * Xh[:, i]) < tol


def test_invert_dense_matches_brute_force_and_oracle():
    A11, A12, A = _pd_jsym(60, 7)
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    s = _solver(kind="dense", A11=A11, A12=A12, nev=5, m=20, mwin=10, tol=1e-10, invert=True)
    st = s.solve()
    ev, X, res = s.pairs()
    s.close()
    bf = np.linalg.eigvalsh(A)[0::2][:5]
    _check(ev, X, mv, 1e-10, bf)
    ref = tj.trlan_jsym(mv, 120, 5, 20, 10, 1e-12, solve=lambda b: np.linalg.solve(A, b))
    assert np.abs(ev - ref["evals"]).max() < 1e-10 * np.abs(bf).max()
    assert st["n_cg_iters"] > 0 and st["n_matvec_inner"] >= st["n_cg_iters"]
    # N_MV counts the A^{-1} applications, as the oracle does
    assert abs(st["n_matvec"] - ref["n_matvec"]) <= 0.25 * ref["n_matvec"] + 10


def test_invert_stencil_4x4x4x4_matches_brute_force():
    dims = (4, 4, 4, 4)
    U, W = inputs.stencil_links(dims, 1)
    n = 6 * inputs.lattice_volume(dims)
    mv = lambda x: jsym.stencil_matvec(U, W, dims, 8.5, 0.3, x)
    A = np.stack([mv(e) for e in np.eye(n, dtype=np.complex128)], axis=1)
    bf = np.linalg.eigvalsh(A)[0::2][:6]
    s = _solver(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W, nev=6, m=24, mwin=12, tol=1e-10,
                invert=True)
    st = s.solve()
    ev, X, res = s.pairs()
    s.close()
    _check(ev, X, mv, 1e-10, bf)
    assert (res < 1e-10).all()


def test_invert_stencil_8x8x8x8_agrees_with_normal_mode():
    """The 8^4 lattice at full size: invert mode finds the same 20 smallest pairs as normal mode."""
    dims = (8, 8, 8, 8)
    U, W = inputs.stencil_links(dims, 1)
    mv = lambda x: jsym.stencil_matvec(U, W, dims, 8.5, 0.3, x)
    out = []
    for inv in (False, True):
        s = _solver(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W, nev=20, m=60, mwin=30, tol=1e-8,
                    invert=inv)
        st = s.solve()
        ev, X, res = s.pairs()
        s.close()
        assert (res < 1e-8).all()
        out.append((ev, X, st))
    (e0, _, s0), (e1, X1, s1) = out
    assert np.abs(e0 - e1).max() < 1e-10 * np.abs(e0).max()
    Xh = X1.cpu().numpy()
    for i in (0, 7, 19):
        assert np.linalg.norm(mv(Xh[:, i]) - e1[i] * Xh[:, i]) < 1e-8
    assert s1["n_restarts"] < s0["n_restarts"]      # A^{-1} separates the small end


def test_invert_plain_trlan_dense():
    A11, A12, A = _pd_jsym(50, 9)
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    s = _solver(kind="dense", A11=A11, A12=A12, nev=8, m=32, mwin=16, tol=1e-10, invert=True, plain_trlan=True)
    s.solve()
    ev, X, res = s.pairs()
    s.close()
    lam = np.linalg.eigvalsh(A)[:8]   # plain TRLAN returns both members of each pair
    _check(ev, X, mv, 1e-10, lam)


def test_invert_indefinite_operator_is_reported():
    from paper_2001_07428_gb300 import binding as B
    A11, A12 = inputs.dense_jsym(40, 3)          # eigenvalues of both signs
    s = _solver(kind="dense", A11=A11, A12=A12, nev=3, m=12, mwin=6, tol=1e-10, invert=True)
    with pytest.raises(B.JTRLanError) as ei:
        s.solve()
    assert ei.value.status == B.JTRLAN_EBREAKDOWN and "positive definite" in str(ei.value)
    s.close()
