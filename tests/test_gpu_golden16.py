"""The 16^4 workload (n = 393,216, nev 50, m 120, mwin 60, residual 1e-8) against the oracle.

tests/golden/stencil_16x16x16x16.json holds the oracle's 50 eigenvalues of this seeded workload (the
CPU FP64 implementation of Algorithms 1 and 2, run to residual 1e-10 by tests/golden/make_golden.py,
which calls nothing but the oracle; a residual r bounds each eigenvalue's error by r).  Plain FP64, the compensated form and the learned-filter form must
each return every one of the 50 within 1e-10 relative, with true residuals below 1e-8 (the
library's FP64 check; sampled pairs recomputed here with the oracle's stencil).
"""
import json
import os

import numpy as np
import pytest

from oracle import jsym
from paper_2001_07428_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "stencil_16x16x16x16.json")


@pytest.fixture(scope="module")
def problem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2001_07428_gb300 import binding
    binding.load()
    g = json.load(open(GOLDEN))
    p = g["params"]
    dims = tuple(p["dims"])
    U, W = inputs.stencil_links(dims, p["seed"])
    return g, p, dims, U, W


@pytest.mark.parametrize("form", ["fp64", "mixed_reorth", "learned"])
def test_16x16x16x16_matches_the_oracle(problem, form):
    from paper_2001_07428_gb300 import learned_filter as LF
    from paper_2001_07428_gb300.solver import JTRLan
    g, p, dims, U, W = problem
    nev, m, mwin, tol = p["nev"], p["m"], p["mwin"], 1e-8
    if form == "learned":
        net = LF.FilterNet.load(device="cuda:0")
        s, _, info = LF.solve_learned(net, U, W, dims, p["m0"], p["kappa"], nev, m, mwin, tol, device="cuda:0")
        assert not info["fallback"]
    else:
        s = JTRLan(kind="stencil", dims=dims, m0=p["m0"], kappa=p["kappa"], U=U, W=W, nev=nev, m=m, mwin=mwin,
                   tol=tol, precision=form, device="cuda:0")
        s.solve()
    ev, X, res = s.pairs()
    s.close()
    assert g["tol"] <= 1e-10
    ref = np.array(g["evals"])
    err = np.abs(ev - ref) / np.abs(ref)
    assert err.max() < 1e-10, f"eigenvalue {err.argmax()}: relative error {err.max():.3e}"
    assert (res < tol).all()
    Xh = X.cpu().numpy()
    for i in (0, nev // 2, nev - 1):
        r = jsym.stencil_matvec(U, W, dims, p["m0"], p["kappa"], Xh[:, i]) - ev[i] * Xh[:, i]
        assert np.linalg.norm(r) < tol
