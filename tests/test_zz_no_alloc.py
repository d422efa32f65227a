"""jtrlan_residual_norms_noalloc: residual norms for callers that cannot allocate device memory.

Such callers (an application whose own caching allocator holds the device memory it may use, code
that must not let cudaMalloc synchronise the device under other streams, a plug-in with no
allocation rights) get the solver's residual kernel with its scratch in a static device array.
This test calls it through the C ABI, twice in a row, and checks it against the residuals that
jtrlan_pairs reports for the same eigenpairs (the existing entry point, same kernels), within the
tolerance of the other parity tests, and against the CPU oracle's matvec.  It lives in a file of
its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from oracle import jsym
from paper_2001_07428_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2001_07428_gb300 import binding
    binding.load()


def _solve_and_noalloc(kind):
    from paper_2001_07428_gb300 import binding as B
    from paper_2001_07428_gb300.solver import JTRLan
    dev = torch.device("cuda:0")
    if kind == "stencil":
        dims = (4, 4, 4, 4)
        U, W = inputs.stencil_links(dims, seed=1)
        Ud, Wd = torch.from_numpy(U).to(dev), torch.from_numpy(W).to(dev)
        op = B.stencil_operator(dims, 8.5, 0.3, Ud.data_ptr(), Wd.data_ptr())
        s = JTRLan("stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W, nev=8, m=30, mwin=16, tol=1e-10,
                   device="cuda:0")
        mv = lambda x: jsym.stencil_matvec(U, W, dims, 8.5, 0.3, x)
        keep = (Ud, Wd)
    else:
        A11, A12 = inputs.dense_jsym(100, 0)
        Ad, Bd = torch.from_numpy(A11).to(dev), torch.from_numpy(A12).to(dev)
        op = B.dense_operator(200, Ad.data_ptr(), Bd.data_ptr())
        s = JTRLan("dense", A11=A11, A12=A12, nev=10, m=30, mwin=15, tol=1e-10, device="cuda:0")
        mv = lambda x: jsym.dense_matvec(A11, A12, x)
        keep = (Ad, Bd)
    s.solve()
    ev, X, res_pairs = s.pairs()
    s.close()
    Xc = X.T.contiguous()          # (nev, n) row-major = n x nev column-major
    n, nev = X.shape
    stream = torch.cuda.current_stream(dev).cuda_stream
    outs = []
    for _ in range(2):             # two calls in a row share the static scratch
        res = np.full(nev, np.nan)
        B.jtrlan_residual_norms_noalloc(op, Xc.data_ptr(), n, nev, ev.ctypes.data_as(ctypes.c_void_p),
                                        res.ctypes.data_as(ctypes.c_void_p), stream)
        outs.append(res)
    del keep
    return ev, Xc.cpu().numpy().T, res_pairs, outs, mv, op


@pytest.mark.parametrize("kind", ["dense", "stencil"])
def test_noalloc_residuals_match_pairs(kind):
    ev, X, res_pairs, outs, mv, _ = _solve_and_noalloc(kind)
    for res in outs:
        assert np.all(np.isfinite(res))
        assert np.allclose(res, res_pairs, rtol=1e-8, atol=1e-15)
    assert np.array_equal(outs[0], outs[1])
    ref = np.array([np.linalg.norm(mv(X[:, i]) - ev[i] * X[:, i]) for i in range(len(ev))])
    assert np.allclose(outs[0], ref, rtol=1e-6, atol=1e-13)


def test_noalloc_leading_dimension_beyond_n():
    """The same columns at a column stride ldx = n + 8 give the same norms, bit for bit."""
    from paper_2001_07428_gb300 import binding as B
    dev = torch.device("cuda:0")
    A11, A12 = inputs.dense_jsym(100, 0)
    Ad, Bd = torch.from_numpy(A11).to(dev), torch.from_numpy(A12).to(dev)
    op = B.dense_operator(200, Ad.data_ptr(), Bd.data_ptr())
    n, ncols, ldx = 200, 6, 208
    rng = np.random.default_rng(5)
    X = rng.standard_normal((ncols, n)) + 1j * rng.standard_normal((ncols, n))
    lam = rng.standard_normal(ncols)
    Xd = torch.from_numpy(X).to(dev)                          # column i at offset i * n
    Xs = torch.zeros((ncols, ldx), dtype=torch.complex128, device=dev)
    Xs[:, :n] = Xd                                            # column i at offset i * ldx
    stream = torch.cuda.current_stream(dev).cuda_stream
    out = []
    for ptr, ld in ((Xd.data_ptr(), n), (Xs.data_ptr(), ldx)):
        res = np.full(ncols, np.nan)
        B.jtrlan_residual_norms_noalloc(op, ptr, ld, ncols, lam.ctypes.data_as(ctypes.c_void_p),
                                        res.ctypes.data_as(ctypes.c_void_p), stream)
        out.append(res)
    assert np.array_equal(out[0], out[1])
    ref = [np.linalg.norm(jsym.dense_matvec(A11, A12, X[i]) - lam[i] * X[i]) for i in range(ncols)]
    assert np.allclose(out[0], ref, rtol=1e-12)


def _expect_einval(op, X, ld, ncols, word):
    """The call must fail with JTRLAN_EINVAL naming `word`; every pointer passed is a real buffer of
    the stated size, so a regression in the checks could not reach a wild address."""
    from paper_2001_07428_gb300 import binding as B
    lam = np.zeros(ncols)
    res = np.zeros(ncols)
    with pytest.raises(B.JTRLanError) as ei:
        B.jtrlan_residual_norms_noalloc(op, X.data_ptr(), ld, ncols, lam.ctypes.data_as(ctypes.c_void_p),
                                        res.ctypes.data_as(ctypes.c_void_p),
                                        torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == B.JTRLAN_EINVAL
    assert word in str(ei.value)


def test_noalloc_rejects_partials_beyond_the_limit():
    from paper_2001_07428_gb300 import binding as B
    dev = torch.device("cuda:0")
    dims = (8, 8, 8, 8)                               # 384 blocks per product
    U, W = inputs.stencil_links(dims, seed=1)
    Ud, Wd = torch.from_numpy(U).to(dev), torch.from_numpy(W).to(dev)
    op = B.stencil_operator(dims, 8.5, 0.3, Ud.data_ptr(), Wd.data_ptr())
    ncols = B.NOALLOC_MAX_PARTIALS // 384 + 1
    X = torch.zeros((ncols, op.n), dtype=torch.complex128, device=dev)
    _expect_einval(op, X, op.n, ncols, "MAX_PARTIALS")


def test_noalloc_rejects_columns_beyond_the_limit():
    from paper_2001_07428_gb300 import binding as B
    dev = torch.device("cuda:0")
    A11, A12 = inputs.dense_jsym(8, 0)                # n = 16: one block per product
    Ad, Bd = torch.from_numpy(A11).to(dev), torch.from_numpy(A12).to(dev)
    op = B.dense_operator(16, Ad.data_ptr(), Bd.data_ptr())
    ncols = B.NOALLOC_MAX_COLS + 1
    X = torch.zeros((ncols, 16), dtype=torch.complex128, device=dev)
    _expect_einval(op, X, 16, ncols, "MAX_COLS")


def test_noalloc_rejects_complex64_operators():
    from paper_2001_07428_gb300 import binding as B
    dev = torch.device("cuda:0")
    A11, A12 = inputs.dense_jsym(8, 0)
    Ad = torch.from_numpy(A11.astype(np.complex64)).to(dev)
    Bd = torch.from_numpy(A12.astype(np.complex64)).to(dev)
    op = B.dense_operator(16, Ad.data_ptr(), Bd.data_ptr(), dtype=B.JTRLAN_C64)
    X = torch.zeros((2, 16), dtype=torch.complex128, device=dev)
    _expect_einval(op, X, 16, 2, "complex128")
