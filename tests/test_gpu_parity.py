"""GPU parity: the CUDA path through the C ABI against the CPU FP64 oracle on the same seeded inputs.

Tolerances: eigenvalues within 1e-10 relative of the oracle (run to 1e-12); true residuals
||A x - lambda x|| / ||x|| below the solve tolerance, recomputed here on the CPU with the oracle's
matvec; the matvec itself element by element within 1e-13 relative to max|y| (FP64 summation
order differs).  Eigenvectors are compared as 2-D pair spaces span{x, J x*}: any unitary mix of a
J pair is an equally correct answer.
"""
import json
import os

import numpy as np
import pytest

from oracle import jsym
from oracle import trlan_jsym as tj
from paper_2001_07428_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2001_07428_gb300 import binding
    binding.load()


def _solver(**kw):
    from paper_2001_07428_gb300.solver import JTRLan
    return JTRLan(**kw, device="cuda:0")


def _check_pairs(ev, X, mv, tol, ev_ref=None, X_ref=None, rel=1e-10):
    Xh = X.cpu().numpy()
    nev = len(ev)
    if ev_ref is not None:
        err = np.abs(ev - ev_ref) / np.maximum(np.abs(ev_ref), 1e-300)
        assert err.max() < rel, f"eigenvalue rel err {err.max():.3e}"
    G = Xh.conj().T @ Xh
    assert np.abs(G - np.eye(nev)).max() < 1e-10                       # X^H X = I
    Y = np.stack([jsym.pair(Xh[:, i]) for i in range(nev)], axis=1)
    assert np.abs(Y.conj().T @ Xh).max() < 1e-10                       # (J X*)^H X = O
    for i in range(nev):
        r = mv(Xh[:, i]) - ev[i] * Xh[:, i]
        assert np.linalg.norm(r) / np.linalg.norm(Xh[:, i]) < tol, f"residual {i}"
    if X_ref is not None:  # each x_i lies in the oracle's pair space span{x_i, J x_i^*}
        for i in range(nev):
            Q = np.stack([X_ref[:, i], jsym.pair(X_ref[:, i])], axis=1)
            resid = Xh[:, i] - Q @ (Q.conj().T @ Xh[:, i])
            assert np.linalg.norm(resid) < 1e-6


# ----------------------------------------------------------------------------- matvec
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 5, 2, 7), (8, 8, 8, 8), (1, 2, 3, 4)])
def test_stencil_apply_matches_oracle(dims):
    U, W = inputs.stencil_links(dims, seed=3)
    n = 6 * inputs.lattice_volume(dims)
    s = _solver(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W, nev=1, m=2, mwin=1, tol=1e-8)
    for seed in range(3):
        x = inputs.random_vector(n, seed)
        y = s.apply(torch.from_numpy(x)).cpu().numpy()
        ref = jsym.stencil_matvec(U, W, dims, 8.5, 0.3, x)
        assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
    s.close()


@pytest.mark.parametrize("h", [8, 100, 257])
def test_dense_apply_matches_oracle(h):
    A11, A12 = inputs.dense_jsym(h, seed=h)
    s = _solver(kind="dense", A11=A11, A12=A12, nev=1, m=2, mwin=1, tol=1e-8)
    x = inputs.random_vector(2 * h, 7)
    y = s.apply(torch.from_numpy(x)).cpu().numpy()
    ref = jsym.dense_matvec(A11, A12, x)
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
    s.close()


# ----------------------------------------------------------------------------- full solves
def test_dense_n200_matches_oracle_and_brute_force():
    w = inputs.WORKLOADS["dense_n200"]
    A11, A12 = inputs.dense_jsym(w["n"] // 2, w["seed"])
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    ref = tj.trlan_jsym(mv, w["n"], w["nev"], w["m"], w["mwin"], 1e-12)
    brute = np.linalg.eigvalsh(jsym.assemble_block_form(A11, A12))[0::2][: w["nev"]]
    s = _solver(kind="dense", A11=A11, A12=A12, nev=w["nev"], m=w["m"], mwin=w["mwin"], tol=1e-10,
                check_jsym=True)
    stats = s.solve()
    ev, X, res = s.pairs(with_partners=True)
    s.close()
    _check_pairs(ev, X[:, : w["nev"]], mv, 1e-10, ref["evals"], ref["X"])
    assert np.abs(ev - brute).max() < 1e-10 * np.abs(brute).max()
    assert np.all(res < 1e-10)
    # partners (eq. (2)): column nev + i is J x_i^*
    Xh = X.cpu().numpy()
    for i in range(w["nev"]):
        assert np.allclose(Xh[:, w["nev"] + i], jsym.pair(Xh[:, i]), atol=0)
    m, mwin, nev, nc = w["m"], w["mwin"], w["nev"], stats["n_restarts"]
    assert m + (m - mwin - nev) * (nc - 1) <= stats["n_matvec"] <= m + (m - mwin) * (nc - 1)  # eq. (30)


def test_dense_largest():
    A11, A12 = inputs.dense_jsym(80, 3)
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    ref = tj.trlan_jsym(mv, 160, 6, 24, 12, 1e-12, which="largest")
    s = _solver(kind="dense", A11=A11, A12=A12, nev=6, m=24, mwin=12, tol=1e-10, which="largest")
    s.solve()
    ev, X, _ = s.pairs()
    s.close()
    assert np.all(np.diff(ev) <= 0)
    _check_pairs(ev, X, mv, 1e-10, ref["evals"], ref["X"])


@pytest.mark.parametrize("dims,nev,m,mwin", [((4, 4, 4, 4), 10, 40, 20), ((3, 5, 2, 7), 8, 30, 16)])
def test_stencil_small_matches_oracle(dims, nev, m, mwin):
    U, W = inputs.stencil_links(dims, seed=1)
    n = 6 * inputs.lattice_volume(dims)
    mv = lambda x: jsym.stencil_matvec(U, W, dims, 8.5, 0.3, x)
    ref = tj.trlan_jsym(mv, n, nev, m, mwin, 1e-12)
    s = _solver(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W, nev=nev, m=m, mwin=mwin, tol=1e-10)
    s.solve()
    ev, X, _ = s.pairs()
    s.close()
    _check_pairs(ev, X, mv, 1e-10, ref["evals"], ref["X"])


def test_stencil_8x8x8x8_matches_golden():
    """The 8^4 workload (n = 24,576, nev = 20, m = 60) against the stored oracle eigenvalues."""
    g = json.load(open(os.path.join(HERE, "golden", "stencil_8x8x8x8.json")))
    p = g["params"]
    dims = tuple(p["dims"])
    U, W = inputs.stencil_links(dims, p["seed"])
    mv = lambda x: jsym.stencil_matvec(U, W, dims, p["m0"], p["kappa"], x)
    s = _solver(kind="stencil", dims=dims, m0=p["m0"], kappa=p["kappa"], U=U, W=W, nev=p["nev"], m=p["m"],
                mwin=p["mwin"], tol=1e-8)
    stats = s.solve()
    ev, X, res = s.pairs()
    s.close()
    _check_pairs(ev, X, mv, 1e-8, np.array(g["evals"]))
    assert np.all(res < 1e-8)
    m, mwin, nev, nc = p["m"], p["mwin"], p["nev"], stats["n_restarts"]
    assert m + (m - mwin - nev) * (nc - 1) <= stats["n_matvec"] <= m + (m - mwin) * (nc - 1)


def test_constant_links_closed_form_and_breakdown():
    from paper_2001_07428_gb300 import binding as B
    from tests import closed_form as cf
    dims = (6, 6, 6, 6)
    U, W, U0, W0 = inputs.constant_links(dims, seed=21)
    n = 6 * 6 ** 4
    exact = cf.constant_link_spectrum(U0, W0, dims, 8.5, 0.3)[0::2]
    # v1 = (1,...,1) spans an invariant subspace here: the library must report the breakdown
    s = _solver(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W, nev=6, m=40, mwin=12, tol=1e-10)
    with pytest.raises(B.JTRLanError) as ei:
        s.solve()
    assert ei.value.status == B.JTRLAN_EBREAKDOWN
    s.close()
    v1 = inputs.random_vector(n, 5)
    s = _solver(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W, nev=6, m=40, mwin=12, tol=1e-10, v1=v1)
    s.solve()
    ev, X, _ = s.pairs()
    s.close()
    mv = lambda x: jsym.stencil_matvec(U, W, dims, 8.5, 0.3, x)
    _check_pairs(ev, X, mv, 1e-10, exact[:6])


# ----------------------------------------------------------------------------- statuses
def test_lemma1_check_rejects_broken_operator():
    from paper_2001_07428_gb300 import binding as B
    A11, A12 = inputs.dense_jsym(50, 2)
    A12_bad = A12 + 0.1 * np.eye(50)            # no longer skew-symmetric: not J-symmetric
    with pytest.raises(B.JTRLanError) as ei:
        _solver(kind="dense", A11=A11, A12=A12_bad, nev=4, m=12, mwin=4, tol=1e-8, check_jsym=True)
    assert ei.value.status == B.JTRLAN_ENOTJSYM


def test_no_convergence_status():
    from paper_2001_07428_gb300 import binding as B
    A11, A12 = inputs.dense_jsym(100, 0)
    s = _solver(kind="dense", A11=A11, A12=A12, nev=10, m=12, mwin=1, tol=1e-14, max_restarts=2)
    with pytest.raises(B.JTRLanError) as ei:
        s.solve()
    assert ei.value.status == B.JTRLAN_ENOCONV
    with pytest.raises(B.JTRLanError) as ei:
        s.pairs()
    assert ei.value.status == B.JTRLAN_ESTATE
    s.close()


def test_solve_twice_is_reproducible():
    A11, A12 = inputs.dense_jsym(100, 0)
    s = _solver(kind="dense", A11=A11, A12=A12, nev=10, m=30, mwin=15, tol=1e-10)
    st1 = s.solve(); ev1, X1, _ = s.pairs()
    st2 = s.solve(); ev2, X2, _ = s.pairs()
    s.close()
    assert st1["n_matvec"] == st2["n_matvec"]
    assert np.array_equal(ev1, ev2)
    assert torch.equal(X1, X2)


# ----------------------------------------------------------------------------- mixed precision
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 8, 8, 8)])
def test_fp32_apply_matches_oracle(dims):
    """The FP32 operator of a mixed context: within FP32 rounding of the FP64 oracle."""
    U, W = inputs.stencil_links(dims, seed=3)
    n = 6 * inputs.lattice_volume(dims)
    s = _solver(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W, nev=1, m=2, mwin=1, tol=1e-8,
                precision="mixed")
    x = inputs.random_vector(n, 0)
    y = s.apply(torch.from_numpy(x)).cpu().numpy().astype(np.complex128)
    ref = jsym.stencil_matvec(U, W, dims, 8.5, 0.3, x)
    assert np.abs(y - ref).max() <= 2e-6 * np.abs(ref).max()
    s.close()


@pytest.mark.parametrize("precision", ["mixed", "mixed_reorth"])
def test_mixed_dense_n200_matches_oracle(precision):
    w = inputs.WORKLOADS["dense_n200"]
    A11, A12 = inputs.dense_jsym(w["n"] // 2, w["seed"])
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    ref = tj.trlan_jsym(mv, w["n"], w["nev"], w["m"], w["mwin"], 1e-12)
    s = _solver(kind="dense", A11=A11, A12=A12, nev=w["nev"], m=w["m"], mwin=w["mwin"], tol=1e-10,
                precision=precision)
    stats = s.solve()
    ev, X, res = s.pairs()
    s.close()
    if precision == "mixed":
        assert stats["n_matvec_fp32"] > 0 and stats["n_matvec"] > stats["n_matvec_fp32"]
    _check_pairs(ev, X, mv, 1e-10, ref["evals"], ref["X"])


@pytest.mark.parametrize("precision", ["mixed", "mixed_reorth"])
def test_mixed_stencil_8x8x8x8_matches_golden(precision):
    g = json.load(open(os.path.join(HERE, "golden", "stencil_8x8x8x8.json")))
    p = g["params"]
    dims = tuple(p["dims"])
    U, W = inputs.stencil_links(dims, p["seed"])
    mv = lambda x: jsym.stencil_matvec(U, W, dims, p["m0"], p["kappa"], x)
    s = _solver(kind="stencil", dims=dims, m0=p["m0"], kappa=p["kappa"], U=U, W=W, nev=p["nev"], m=p["m"],
                mwin=p["mwin"], tol=1e-8, precision=precision)
    stats = s.solve()
    ev, X, res = s.pairs()
    s.close()
    assert (stats["n_matvec_fp32"] > 0) == (precision == "mixed")
    _check_pairs(ev, X, mv, 1e-8, np.array(g["evals"]))
    assert np.all(res < 1e-8)


def test_mixed_reorth_complex64_links_match_brute_force():
    """Complex64 links are exact in FP32: the compensated products read them as (hi, 0) pairs.  The
    eigenvalues must match brute-force diagonalisation of the operator those links define."""
    dims = (4, 4, 4, 4)
    U, W = inputs.stencil_links(dims, 5)
    U32 = U.astype(np.complex64).astype(np.complex128)
    W32 = W.astype(np.complex64).astype(np.complex128)
    n = 6 * inputs.lattice_volume(dims)
    mv = lambda x: jsym.stencil_matvec(U32, W32, dims, 8.5, 0.3, x)
    A = np.stack([mv(e) for e in np.eye(n, dtype=np.complex128)], axis=1)
    bf = np.linalg.eigvalsh(A)[0::2][:8]
    s = _solver(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U.astype(np.complex64), W=W.astype(np.complex64),
                nev=8, m=30, mwin=15, tol=1e-10, precision="mixed_reorth", links_dtype="c64")
    s.solve()
    ev, X, res = s.pairs()
    s.close()
    assert np.abs(ev - bf).max() < 1e-10 * np.abs(bf).max()
    Xh = X.cpu().numpy()
    for i in range(8):
        assert np.linalg.norm(mv(Xh[:, i]) - ev[i] * Xh[:, i]) < 1e-10
