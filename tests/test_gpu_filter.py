"""GPU parity of the filtered form and of the network that predicts its coefficients, through the C ABI.

* p(A) x (FP32 operator and recurrence) against the FP64 oracle recurrence: within 2e-5 of max|y|
  (FP32 rounding grows at most like the degree times the unit roundoff along the recurrence).
* The filtered mixed solve against the oracle's unfiltered eigenpairs: eigenvalues within 1e-10
  relative, true residuals below tol (the filter changes the path, not the answer).
* The spectral window from jtrlan_bounds brackets the brute-force extremes as documented.
* Damped step coefficients against the oracle formula: within 1e-6 (FP32 output).
* The MLP forward pass, gradient and one Adam step against the FP64 oracle with the same
  parameters: within FP32 tolerances (1e-5 relative on outputs, 1e-4 of max|g| on gradients).
"""
import numpy as np
import pytest

from oracle import filter as flt
from oracle import jsym
from oracle import mlp as omlp
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


def _stencil(dims, seed, m0=8.5, kappa=0.3):
    U, W = inputs.stencil_links(dims, seed)
    return U, W, lambda x: jsym.stencil_matvec(U, W, dims, m0, kappa, x)


def _solver(**kw):
    from paper_2001_07428_gb300.solver import JTRLan
    return JTRLan(**kw, device="cuda:0")


# ----------------------------------------------------------------------------- p(A) x
@pytest.mark.parametrize("kind,degree", [("dense", 1), ("dense", 17), ("stencil", 64)])
def test_filter_apply_matches_oracle(kind, degree):
    rng = np.random.default_rng(degree)
    g = rng.standard_normal(degree + 1) / np.sqrt(degree + 1)
    if kind == "dense":
        A11, A12 = inputs.dense_jsym(70, 11)
        mv = lambda x: jsym.dense_matvec(A11, A12, x)
        lam = np.linalg.eigvalsh(jsym.assemble_block_form(A11, A12))
        win = (lam[0] - 0.5, lam[-1] + 0.5)
        s = _solver(kind="dense", A11=A11, A12=A12, nev=4, m=16, mwin=8, tol=1e-8, precision="mixed",
                    filter_coeffs=g, filter_window=win)
        n = 140
    else:
        dims = (4, 4, 4, 4)
        U, W, mv = _stencil(dims, 5)
        win = (8.5 - 9.0, 8.5 + 9.0)                       # |A - m0| <= 8 + 8 kappa |W| for these links
        s = _solver(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W, nev=4, m=16, mwin=8, tol=1e-8,
                    precision="mixed", filter_coeffs=g, filter_window=win)
        n = 6 * 256
    x = inputs.random_vector(n, 3)
    y = s.apply_filter(torch.from_numpy(x)).cpu().numpy().astype(np.complex128)
    ref = flt.apply_poly(mv, x.astype(np.complex64).astype(np.complex128), g, *win)
    assert np.abs(y - ref).max() < 2e-5 * np.abs(ref).max()
    s.close()


# ----------------------------------------------------------------------------- certifying filter
# The certifying phase's p(A) x through jtrlan_apply_filter, against the oracle's FP64 recurrence on
# the same links.  Tolerances from the arithmetic, relative to max|p(A) x|:
#   * mixed_reorth stencil: each Chebyshev step fused into the compensated-FP32 product whose sums are
#     carried at a fixed bias per direction, about 2^-40.8 of sum |a| |x| a product (an exact
#     emulation of the sequence: the worst of 300 random 48-term sums); over d steps of the recurrence
#     the errors add up to about d times that, held to 10 d 2^-40.8 (3.2e-10 at d = 64; the FP32 case
#     above is held to 5 d u the same way);
#   * FP64: FP64 products and recurrence, 10 d 2^-52.
# Lattices (3, 5, 2, 7) (210 sites: four 64-site blocks, the last ragged) and 8^4 (64 blocks).
@pytest.mark.parametrize("dims,links,degree,precision", [
    ((3, 5, 2, 7), "c64", 1, "mixed_reorth"), ((3, 5, 2, 7), "c64", 64, "mixed_reorth"),
    ((3, 5, 2, 7), "c128", 64, "mixed_reorth"), ((8, 8, 8, 8), "c64", 64, "mixed_reorth"),
    ((8, 8, 8, 8), "c128", 17, "mixed_reorth"), ((3, 5, 2, 7), "c128", 64, "fp64")])
def test_certifying_filter_product_matches_oracle(dims, links, degree, precision):
    U, W = inputs.stencil_links(dims, 7)
    if links == "c64":                                   # the kernels read these links exactly
        U = U.astype(np.complex64).astype(np.complex128)
        W = W.astype(np.complex64).astype(np.complex128)
    mv = lambda x: jsym.stencil_matvec(U, W, dims, 8.5, 0.3, x)
    n = 6 * int(np.prod(dims))
    probe = _solver(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W, nev=2, m=40, mwin=4, tol=1e-8,
                    precision=precision, links_dtype=links)
    lo, hi = probe.bounds(30)
    probe.close()
    win = (lo - 0.05 * (hi - lo), hi + 0.05 * (hi - lo))
    rng = np.random.default_rng(100 + degree)
    g = rng.standard_normal(degree + 1) / np.sqrt(degree + 1)
    s = _solver(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W, nev=2, m=16, mwin=4, tol=1e-8,
                precision=precision, links_dtype=links, filter_final_coeffs=g, filter_window=win)
    x = inputs.random_vector(n, 11)
    y = s.apply_filter(torch.from_numpy(x))
    assert y.dtype == torch.complex128
    y = y.cpu().numpy()
    ref = flt.apply_poly(mv, x, g, *win)
    u = 2.0 ** -40.8 if precision == "mixed_reorth" else 2.0 ** -52
    assert np.abs(y - ref).max() < 10 * degree * u * np.abs(ref).max()
    s.close()


@pytest.mark.parametrize("precision", ["mixed_reorth", "fp64"])
def test_certifying_filter_product_on_a_dense_operator(precision):
    """The dense operator keeps the FP64 product in every form, so p(A) x comes out of FP64 products
    and FP64 recurrence steps: within 10 d 2^-52 of max|p(A) x|."""
    A11, A12 = inputs.dense_jsym(100, 5)
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    lam = np.linalg.eigvalsh(jsym.assemble_block_form(A11, A12))
    win = (lam[0] - 0.5, lam[-1] + 0.5)
    degree = 40
    g = np.random.default_rng(7).standard_normal(degree + 1) / np.sqrt(degree + 1)
    s = _solver(kind="dense", A11=A11, A12=A12, nev=4, m=16, mwin=8, tol=1e-8, precision=precision,
                filter_final_coeffs=g, filter_window=win)
    x = inputs.random_vector(200, 12)
    y = s.apply_filter(torch.from_numpy(x))
    assert y.dtype == torch.complex128
    ref = flt.apply_poly(mv, x, g, *win)
    assert np.abs(y.cpu().numpy() - ref).max() < 10 * degree * 2.0 ** -52 * np.abs(ref).max()
    s.close()


# ----------------------------------------------------------------------------- filtered solve
@pytest.mark.parametrize("kind", ["dense", "stencil"])
def test_filtered_solve_matches_unfiltered_oracle(kind):
    nev, m, mwin, tol = 6, 24, 12, 1e-9
    if kind == "dense":
        A11, A12 = inputs.dense_jsym(100, 0)
        mv = lambda x: jsym.dense_matvec(A11, A12, x)
        n, kw = 200, dict(kind="dense", A11=A11, A12=A12)
    else:
        dims = (4, 4, 4, 4)
        U, W, mv = _stencil(dims, 1)
        n, kw = 6 * 256, dict(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W)
    ref = tj.trlan_jsym(mv, n, nev + 1, m, mwin, 1e-12)
    probe = _solver(nev=nev, m=m, mwin=mwin, tol=tol, precision="mixed", **kw)
    lo, hi = probe.bounds(20)
    probe.close()
    tau = flt.cut_to_tau(0.5 * (ref["evals"][nev - 1] + ref["evals"][nev]), lo, hi)
    g = flt.damped_step_coeffs(tau, 32)
    s = _solver(nev=nev, m=m, mwin=mwin, tol=tol, precision="mixed", filter_coeffs=g, filter_window=(lo, hi), **kw)
    st = s.solve()
    ev, X, res = s.pairs()
    assert (np.abs(ev - ref["evals"][:nev]) / np.abs(ref["evals"][:nev])).max() < 1e-10
    Xh = X.cpu().numpy()
    for i in range(nev):
        assert np.linalg.norm(mv(Xh[:, i]) - ev[i] * Xh[:, i]) < tol
    assert st["n_matvec_fp32"] > 0 and st["n_restarts_fp32"] >= 1
    s.close()


@pytest.mark.parametrize("kind,precision", [("dense", "fp64"), ("dense", "mixed_reorth"), ("stencil", "fp64"),
                                            ("stencil", "mixed_reorth")])
def test_certified_filtered_solve_matches_oracle(kind, precision):
    """The certifying phase on B = p(A) (degree 16): pairs accepted by A's true residual at x^H A x."""
    nev, m, mwin, tol = 6, 24, 12, 1e-9
    if kind == "dense":
        A11, A12 = inputs.dense_jsym(100, 0)
        mv = lambda x: jsym.dense_matvec(A11, A12, x)
        n, kw = 200, dict(kind="dense", A11=A11, A12=A12)
    else:
        dims = (4, 4, 4, 4)
        U, W, mv = _stencil(dims, 1)
        n, kw = 6 * 256, dict(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W)
    ref = tj.trlan_jsym(mv, n, nev + 1, m, mwin, 1e-12)
    probe = _solver(nev=nev, m=m, mwin=mwin, tol=tol, precision=precision, **kw)
    lo, hi = probe.bounds(20)
    probe.close()
    a = lo - 0.02 * (hi - lo)
    tau = flt.cut_to_tau(0.5 * (ref["evals"][nev - 1] + ref["evals"][nev]), a, hi)
    g = flt.damped_step_coeffs(tau, 16)
    s = _solver(nev=nev, m=m, mwin=mwin, tol=tol, precision=precision, filter_final_coeffs=g, filter_window=(a, hi),
                **kw)
    st = s.solve()
    ev, X, res = s.pairs()
    assert (np.abs(ev - ref["evals"][:nev]) / np.abs(ref["evals"][:nev])).max() < 1e-10
    assert (np.diff(ev) > 0).all()                     # reported as eigenvalues of A, ascending
    Xh = X.cpu().numpy()
    for i in range(nev):
        assert np.linalg.norm(mv(Xh[:, i]) - ev[i] * Xh[:, i]) < tol
    assert np.abs(Xh.conj().T @ Xh - np.eye(nev)).max() < 1e-10
    assert st["n_matvec"] % 16 == 0                     # 16 products of A per Lanczos step
    s.close()


def test_bounds_bracket_the_spectrum():
    A11, A12 = inputs.dense_jsym(150, 6)
    lam = np.linalg.eigvalsh(jsym.assemble_block_form(A11, A12))
    for prec in ("fp64", "mixed"):
        s = _solver(kind="dense", A11=A11, A12=A12, nev=4, m=30, mwin=8, tol=1e-8, precision=prec)
        lo, hi = s.bounds(24)
        s.close()
        assert abs(lo - lam[0]) < 0.25 * (lam[-1] - lam[0])               # Ritz value less its residual bound
        assert hi >= lam[-1] - 1e-5                                        # Ritz value + beta


def test_damped_step_kernel_matches_oracle():
    from paper_2001_07428_gb300 import binding as B
    taus = np.array([-0.95, -0.4, 0.0, 0.3, 0.99])
    td = torch.from_numpy(taus).cuda()
    out = torch.empty((5, 65), dtype=torch.float32, device="cuda")
    B.jtrlan_damped_step(td.data_ptr(), 5, 64, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    got = out.cpu().numpy()
    for i, t in enumerate(taus):
        assert np.abs(got[i] - flt.damped_step_coeffs(t, 64)).max() < 1e-6


# ----------------------------------------------------------------------------- the network
F, H, O = 6, 128, 65


def _net(seed=3):
    from paper_2001_07428_gb300 import binding as B
    return B, B.jtrlan_mlp_create(F, H, O, seed, torch.cuda.current_stream().cuda_stream)


def _params(B, net):
    import ctypes
    th = np.zeros(B.jtrlan_mlp_param_count(F, H, O), dtype=np.float32)
    B.jtrlan_mlp_get_params(net, th.ctypes.data_as(ctypes.c_void_p))
    return th


def test_mlp_init_is_glorot_uniform():
    B, net = _net(7)
    th = _params(B, net)
    W1, b1, W2, b2, W3, b3 = omlp.unpack(th.astype(np.float64), F, H, O)
    assert (b1 == 0).all() and (b2 == 0).all() and (b3 == 0).all()
    for W, fi, fo in ((W1, F, H), (W2, H, H), (W3, H, O)):
        lim = np.sqrt(6.0 / (fi + fo))
        assert np.abs(W).max() <= lim and np.abs(W).max() > 0.9 * lim
        assert abs(W.std() - lim / np.sqrt(3.0)) < 0.1 * lim        # uniform on [-lim, lim]
    B.jtrlan_mlp_destroy(net)


@pytest.mark.parametrize("N", [1, 37, 300])
def test_mlp_forward_and_gradient_match_oracle(N):
    import ctypes
    B, net = _net(5)
    rng = np.random.default_rng(N)
    X = rng.standard_normal((N, F)).astype(np.float32)
    T = rng.standard_normal((N, O)).astype(np.float32) * 0.3
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    Yd = torch.empty((N, O), dtype=torch.float32, device="cuda")
    B.jtrlan_mlp_forward(net, Xd.data_ptr(), N, Yd.data_ptr())
    torch.cuda.synchronize()
    th = _params(B, net).astype(np.float64)
    Yref, _, _ = omlp.forward(th, X, F, H, O)
    assert np.abs(Yd.cpu().numpy() - Yref).max() < 1e-5 * max(1.0, np.abs(Yref).max())
    g = np.zeros(th.size, dtype=np.float32)
    loss = B.jtrlan_mlp_gradient(net, Xd.data_ptr(), Td.data_ptr(), N, g.ctypes.data_as(ctypes.c_void_p))
    Lref, gref = omlp.gradient(th, X, T, F, H, O)
    assert abs(loss - Lref) < 1e-5 * max(1.0, Lref)
    assert np.abs(g - gref).max() < 1e-4 * np.abs(gref).max()
    B.jtrlan_mlp_destroy(net)


def test_mlp_adam_step_matches_oracle_and_training_reduces_loss():
    import ctypes
    B, net = _net(9)
    rng = np.random.default_rng(2)
    N = 256
    X = rng.standard_normal((N, F)).astype(np.float32)
    T = np.tanh(X @ rng.standard_normal((F, O))).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    th0 = _params(B, net).astype(np.float64)
    hist = np.zeros(1, dtype=np.float32)
    B.jtrlan_mlp_train(net, Xd.data_ptr(), Td.data_ptr(), N, 1, 1e-3, hist.ctypes.data_as(ctypes.c_void_p))
    th1 = _params(B, net).astype(np.float64)
    L0, g0 = omlp.gradient(th0, X, T, F, H, O)
    ref1, _, _ = omlp.adam_step(th0, g0, np.zeros_like(th0), np.zeros_like(th0), 1, 1e-3)
    assert abs(hist[0] - L0) < 1e-5 * max(1.0, L0)
    # the first step moves each parameter by lr sign(g) unless |g| is at the FP32 noise floor
    big = np.abs(g0) > 1e-3 * np.abs(g0).max()
    assert np.abs(th1 - ref1)[big].max() < 1e-6
    hist = np.zeros(400, dtype=np.float32)
    B.jtrlan_mlp_train(net, Xd.data_ptr(), Td.data_ptr(), N, 400, 1e-3, hist.ctypes.data_as(ctypes.c_void_p))
    assert hist[-1] < 0.2 * L0 and np.all(np.isfinite(hist))
    B.jtrlan_mlp_destroy(net)
