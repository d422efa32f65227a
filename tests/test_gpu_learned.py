"""What the trained filter network gains over the method without it (GPU, through the C ABI).

* On held-out plain runs the trained network places the filter's cut within 0.005 of the window
  (median), an untrained one nowhere near it.
* On a held-out 12^4 problem (nev = 100, m = 200, residual 1e-8) the learned-filter solve returns the
  same eigenpairs as the unfiltered solve (eigenvalues within 1e-10 relative; residuals recomputed with
  the oracle's stencil below tol) in under half its time and outer iterations.
"""
import json
import time

import numpy as np
import pytest

from oracle import jsym
from paper_2001_07428_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def LF():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2001_07428_gb300 import learned_filter
    return learned_filter


def _held_out(LF):
    records = [r for r in json.load(open(LF.RUNS)) if r["i"] % 8 == 7]
    X, taus = [], []
    for r in records:
        a, b = LF.window(r["lo"], r["hi"])
        for nev in LF.NEV_GRID:
            X.append(LF.features(r["lo"], r["hi"], r["m0"], r["kappa"], nev, r["sites"]))
            taus.append(LF.cut_tau(np.asarray(r["ev"]), nev, a, b))
    return np.stack(X), np.asarray(taus)


def _tau(g):
    return np.cos(np.pi * (1.0 - g[:, 0]))


def test_trained_network_places_the_cut_on_held_out_runs(LF):
    X, taus = _held_out(LF)
    trained = LF.FilterNet.load()
    err = np.abs(_tau(trained.predict(X)) - taus)
    untrained = LF.FilterNet(seed=123)
    err0 = np.abs(_tau(untrained.predict(X)) - taus)
    assert np.median(err) < 0.005 and err.max() < 0.05
    assert np.median(err0) > 10 * np.median(err)


def test_learned_filter_gains_over_the_unfiltered_method(LF):
    from paper_2001_07428_gb300.solver import JTRLan
    dims, m0, kappa, seed = (12, 12, 12, 12), 9.1, 0.3, 4244       # not among the training runs
    nev, m, mwin, tol = 100, 200, 100, 1e-8
    U, W = inputs.stencil_links(dims, seed)
    net = LF.FilterNet.load()
    plain = JTRLan(kind="stencil", dims=dims, m0=m0, kappa=kappa, U=U, W=W, nev=nev, m=m, mwin=mwin, tol=tol,
                   precision="mixed_reorth", device="cuda:0")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st0 = plain.solve()
    t_plain = time.perf_counter() - t0
    ev0, _, _ = plain.pairs()
    plain.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s, st, info = LF.solve_learned(net, U, W, dims, m0, kappa, nev, m, mwin, tol, device="cuda:0")
    t_learned = time.perf_counter() - t0                           # includes the bounds estimate and inference
    ev, X, res = s.pairs()
    s.close()
    assert not info["fallback"]
    assert (np.abs(ev - ev0) / np.abs(ev0)).max() < 1e-10
    Xh = X.cpu().numpy()
    for i in (0, nev // 2, nev - 1):
        r = jsym.stencil_matvec(U, W, dims, m0, kappa, Xh[:, i]) - ev[i] * Xh[:, i]
        assert np.linalg.norm(r) < tol
    assert st["n_restarts"] < st0["n_restarts"] / 2
    assert t_learned < 0.5 * t_plain, (t_learned, t_plain)


def test_filter_set_on_a_context_matches_one_created_with_it(LF):
    """jtrlan_set_filter on a context created without a filter (bounds on that context, then the
    network) gives the same solve, bit for bit, as a context created with those coefficients; the
    eigenvalues agree with the unfiltered solve; a second call replaces the filter and clears the
    pairs until the next solve."""
    from paper_2001_07428_gb300 import binding as B
    from paper_2001_07428_gb300.solver import JTRLan
    dims, nev, m, mwin, tol = (8, 8, 8, 8), 20, 60, 30, 1e-8
    U, W = inputs.stencil_links(dims, 1)
    kw = dict(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W, nev=nev, m=m, mwin=mwin, tol=tol,
              precision="mixed_reorth", device="cuda:0")
    net = LF.FilterNet.load()
    s = JTRLan(**kw)
    g, win, _ = LF.filter_on_context(net, s.ctx, 8.5, 0.3, nev, 4096)
    s.solve()
    ev1, X1, res1 = s.pairs()
    ref = JTRLan(filter_final_coeffs=g, filter_window=win, **kw)
    ref.solve()
    ev0, _, _ = ref.pairs()
    ref.close()
    assert np.array_equal(ev1, ev0)
    plain = JTRLan(**kw)
    plain.solve()
    evp, _, _ = plain.pairs()
    plain.close()
    assert (np.abs(ev1 - evp) / np.abs(evp)).max() < 1e-10
    assert (res1 < tol).all()
    g2, win2, _ = LF.filter_on_context(net, s.ctx, 8.5, 0.3, nev, 4096)
    assert np.array_equal(g2, g) and win2 == win        # bounds are deterministic
    with pytest.raises(B.JTRLanError) as ei:
        s.pairs()
    assert ei.value.status == B.JTRLAN_ESTATE
    s.solve()
    ev2, _, _ = s.pairs()
    s.close()
    assert np.array_equal(ev2, ev1)
