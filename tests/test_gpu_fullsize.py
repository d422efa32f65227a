"""Full-size checks in the configurations the benchmark times, on sampled outputs the oracle can
recompute one by one (GPU, through the C ABI).

* 16^4 stencil (n = 393,216, nev 50, m 120, mwin 60, residual 1e-8, complex64 links): the chosen
  mixed form returns the eigenvalues of the plain FP64 solve within 1e-10 relative; sampled pairs
  have true residuals below tol (the oracle's stencil), unit norm, and their partners J x* are
  orthogonal to them.
* 24^3 x 48 stencil (n = 3,981,312, nev 100, m 200, mwin 100), the learned-filter form: no fallback;
  sampled pairs have true residuals below tol and eigenvalues equal to their Rayleigh quotients
  x^H A x within 1e-12 relative (the oracle's stencil); eigenvalues ascending.
"""
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


def _links(dims, seed):
    U, W = inputs.stencil_links(dims, seed)
    return U.astype(np.complex64), W.astype(np.complex64)


def _check_sampled(X, ev, mv, picks, tol):
    for i in picks:
        x = X[:, i].cpu().numpy()
        assert abs(np.linalg.norm(x) - 1.0) < 1e-12
        Ax = mv(x)
        assert np.linalg.norm(Ax - ev[i] * x) < tol, (i, np.linalg.norm(Ax - ev[i] * x))
        rq = np.vdot(x, Ax)
        assert abs(rq.imag) < 1e-12 * abs(rq.real)
        assert abs(rq.real - ev[i]) < 1e-12 * abs(ev[i])
        assert abs(np.vdot(jsym.pair(x), x)) < 1e-12              # Lemma 1: J x* is orthogonal to x


def test_16x16x16x16_mixed_matches_fp64():
    from paper_2001_07428_gb300.solver import JTRLan
    dims, nev, m, mwin, tol = (16, 16, 16, 16), 50, 120, 60, 1e-8
    U, W = _links(dims, 1)
    kw = dict(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W, nev=nev, m=m, mwin=mwin, tol=tol,
              links_dtype="c64", device="cuda:0")
    out = {}
    for prec in ("fp64", "mixed_reorth"):
        s = JTRLan(precision=prec, **kw)
        s.solve()
        out[prec] = s.pairs()
        s.close()
    e64, _, r64 = out["fp64"]
    ev, X, res = out["mixed_reorth"]
    assert (r64 < tol).all() and (res < tol).all()
    assert (np.abs(ev - e64) / np.abs(e64)).max() < 1e-10
    U64, W64 = U.astype(np.complex128), W.astype(np.complex128)
    mv = lambda x: jsym.stencil_matvec(U64, W64, dims, 8.5, 0.3, x)
    _check_sampled(X, ev, mv, (0, nev // 2, nev - 1), tol)


def test_24x24x24x48_learned_filter_form():
    from paper_2001_07428_gb300 import learned_filter as LF
    dims, nev, m, mwin, tol = (24, 24, 24, 48), 100, 200, 100, 1e-8
    U, W = _links(dims, 1)
    net = LF.FilterNet.load(device="cuda:0")
    s, st, info = LF.solve_learned(net, U, W, dims, 8.5, 0.3, nev, m, mwin, tol, device="cuda:0",
                                   links_dtype="c64")
    ev, X, res = s.pairs()
    s.close()
    assert not info["fallback"]
    assert (res < tol).all()
    assert (np.diff(ev) >= 0).all()
    U64, W64 = U.astype(np.complex128), W.astype(np.complex128)
    del U, W
    mv = lambda x: jsym.stencil_matvec(U64, W64, dims, 8.5, 0.3, x)
    _check_sampled(X, ev, mv, (0, nev // 2, nev - 1), tol)
