"""The restart rotation out = V Z of a compensated-FP32 (hi, lo) basis through the C ABI
(jtrlan_rotate_df), tensor-core path (0) and CUDA-core path (1), against the plain FP64 product of the
same values (the definition of the step: the kept Ritz vectors of Algorithm 1 are V_m times the
eigenvectors of T_m).

Tolerance: every entry within 2^-46 m max_k |V_rk| max_k |Z_kc| of the FP64 product (the digit
splitting of the tensor-core path is exact to 2^-49 of the row and column maxima per product, and
both paths end in float-float); inputs whose digits are few are reproduced bit-exactly.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2001_07428_gb300 import binding
    binding.load()


def _pack(Vc):
    """(n, m) complex128 -> device (m, n, 4) float32 (re_hi, im_hi, re_lo, im_lo), and the exact
    FP64 values hi + lo."""
    re_hi = Vc.real.astype(np.float32)
    im_hi = Vc.imag.astype(np.float32)
    re_lo = (Vc.real - re_hi).astype(np.float32)
    im_lo = (Vc.imag - im_hi).astype(np.float32)
    P = np.stack([re_hi.T, im_hi.T, re_lo.T, im_lo.T], axis=-1)          # (m, n, 4)
    exact = (re_hi.astype(np.float64) + re_lo) + 1j * (im_hi.astype(np.float64) + im_lo)
    return torch.from_numpy(np.ascontiguousarray(P)).to("cuda:0"), exact


def _rotate(Vd, n, m, Z, path):
    from paper_2001_07428_gb300 import binding as B
    kk = Z.shape[1]
    Zd = torch.from_numpy(np.ascontiguousarray(Z.T)).to("cuda:0")            # column c at Z + c m
    out = torch.empty((kk, n), dtype=torch.complex128, device="cuda:0")
    B.jtrlan_rotate_df(Vd.data_ptr(), n, m, Zd.data_ptr(), kk, out.data_ptr(), path,
                       torch.cuda.current_stream().cuda_stream)
    return out.cpu().numpy().T                                               # (n, kk)


def _bound(Vx, Z):
    """2^-46 m max_k |V_rk| max_k |Z_kc| for the real and imaginary rows separately."""
    m = Vx.shape[1]
    rre = np.abs(Vx.real).max(axis=1)[:, None]
    rim = np.abs(Vx.imag).max(axis=1)[:, None]
    cz = np.abs(Z).max(axis=0)[None, :]
    return 2.0**-46 * m * rre * cz, 2.0**-46 * m * rim * cz


def _check(got, Vx, Z, rows=None):
    Vs = Vx if rows is None else Vx[rows]
    ref = Vs @ Z
    g = got if rows is None else got[rows]
    bre, bim = _bound(Vs, Z)
    assert (np.abs(g.real - ref.real) <= bre).all(), np.max(np.abs(g.real - ref.real) / np.maximum(bre, 1e-300))
    assert (np.abs(g.imag - ref.imag) <= bim).all(), np.max(np.abs(g.imag - ref.imag) / np.maximum(bim, 1e-300))


@pytest.mark.parametrize("path", [0, 1])
def test_few_digit_inputs_are_exact(path):
    # ragged everywhere: 2n = 600 real rows (4 tiles of 128 and 88), m = 45 (3 chunks of 16, the last
    # one 13), kk = 70 (3 column tiles of 32, the last one 6)
    rng = np.random.default_rng(11)
    n, m, kk = 300, 45, 70
    Vc = (rng.integers(-1000, 1001, (n, m)) + 1j * rng.integers(-1000, 1001, (n, m))) * 2.0**-10
    Z = rng.integers(-300, 301, (m, kk)) * 2.0**-9
    Vd, Vx = _pack(Vc)
    got = _rotate(Vd, n, m, Z, path)
    ref = Vx @ Z
    if path == 0:
        assert np.array_equal(got, ref)
    else:
        _check(got, Vx, Z)


@pytest.mark.parametrize("n,m,kk", [(1000, 200, 100), (777, 320, 33), (1, 1, 1), (64, 16, 32), (2049, 61, 45)])
def test_orthonormal_basis_matches_fp64_product(n, m, kk):
    rng = np.random.default_rng(n + 7 * m + kk)
    G = rng.standard_normal((n, min(m, n))) + 1j * rng.standard_normal((n, min(m, n)))
    Q = np.linalg.qr(G)[0] if n >= m else G
    Vc = np.zeros((n, m), dtype=np.complex128)
    Vc[:, : Q.shape[1]] = Q
    Z = np.linalg.qr(rng.standard_normal((m, m)))[0][:, :kk] if kk <= m else rng.standard_normal((m, kk))
    Vd, Vx = _pack(Vc)
    g0 = _rotate(Vd, n, m, Z, 0)
    g1 = _rotate(Vd, n, m, Z, 1)
    _check(g0, Vx, Z)
    _check(g1, Vx, Z)


def test_degenerate_rows_and_columns():
    rng = np.random.default_rng(5)
    n, m, kk = 200, 40, 40
    Vc = (rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))) / np.sqrt(n)
    Vc[3, :] = 0.0                       # zero row (both real and imaginary)
    Vc[4, :] = Vc[4, :].real             # zero imaginary row
    Vc[5, :] *= 1e-30                    # tiny row (2^-100 scale)
    Vc[6, :] *= 1e10                     # large row
    Vc[7, :] = 0.0
    Vc[7, 9] = 2.0**-3                   # a single exact power of two
    Vc[8, :] = np.where(np.arange(m) % 2 == 0, 1.0, 1e-12)   # mixed magnitudes along a row
    Z = np.linalg.qr(rng.standard_normal((m, m)))[0]
    Z[:, 2] = 0.0                        # zero column
    Z[:, 3] *= 1e-20                     # tiny column
    Z[5, 4] = 1.0                        # a column with one dominant entry
    Vd, Vx = _pack(Vc)
    got = _rotate(Vd, n, m, Z, 0)
    _check(got, Vx, Z)
    assert np.array_equal(got[3], np.zeros(kk)) and np.array_equal(got[:, 2], np.zeros(n))
    # beyond FP32 range: the tensor-core path keeps Z in FP64 and scales by exact powers of two
    Z2 = Z.copy()
    Z2[:, 3] *= 1e-180
    Z2[:, 5] *= 1e30                     # large column (2^100 scale, within the |Z| < 2^120 limit)
    _check(_rotate(Vd, n, m, Z2, 0), Vx, Z2)
    # the CUDA-core path multiplies FP32 pairs: the same structure with products inside FP32 range
    Vc[5, :] *= 1e20
    Z[:, 3] *= 1e10
    Vd, Vx = _pack(Vc)
    got = _rotate(Vd, n, m, Z, 1)
    _check(got, Vx, Z)
    assert np.array_equal(got[3], np.zeros(kk)) and np.array_equal(got[:, 2], np.zeros(n))


def test_full_size_sampled_rows():
    """The 16^4 lattice's basis shape (n = 393,216, m = 120, kk = 60), checked on sampled rows."""
    rng = np.random.default_rng(3)
    n, m, kk = 393216, 120, 60
    Vc = (rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))) / np.sqrt(2 * n)
    Z = np.linalg.qr(rng.standard_normal((m, m)))[0][:, :kk]
    Vd, Vx = _pack(Vc)
    del Vc
    got = _rotate(Vd, n, m, Z, 0)
    rows = np.unique(np.r_[0, 1, n - 1, n // 2, rng.choice(n, 4000, replace=False)])
    _check(got, Vx, Z, rows)


def test_solver_rotation_paths_agree():
    """JTRLAN_MIXED_REORTH on the 8^4 stencil with the rotation on the tensor cores and on the CUDA
    cores: the same pairs to the solve tolerance."""
    from oracle import jsym
    from paper_2001_07428_gb300 import inputs
    from paper_2001_07428_gb300.solver import JTRLan
    dims = (8, 8, 8, 8)
    U, W = inputs.stencil_links(dims, 1)
    out = []
    for simt in (False, True):
        s = JTRLan(kind="stencil", dims=dims, m0=8.5, kappa=0.3, U=U, W=W, nev=20, m=60, mwin=20, tol=1e-8,
                   precision="mixed_reorth", rotate_simt=simt, device="cuda:0")
        st = s.solve()
        ev, X, res = s.pairs()
        s.close()
        assert (res < 1e-8).all()
        out.append((ev, X.cpu().numpy(), st))
    (e0, X0, s0), (e1, X1, s1) = out
    assert np.abs(e0 - e1).max() < 1e-10 * np.abs(e0).max()
    mv = lambda x: jsym.stencil_matvec(U, W, dims, 8.5, 0.3, x)
    for i in range(0, 20, 5):
        assert np.linalg.norm(mv(X0[:, i]) - e0[i] * X0[:, i]) < 1e-8


def test_bounded_wait_reports_timeout_and_the_stream_stays_usable():
    """path 2 leaves one accumulator barrier unsignalled: the kernel's bounded wait (about 2 s) runs
    out, it frees its tensor memory and returns, and the call reports JTRLAN_ETIMEOUT; the next call
    on the same stream computes the right product."""
    import time
    from paper_2001_07428_gb300 import binding as B
    rng = np.random.default_rng(21)
    n, m, kk = 4096, 32, 32
    Vc = (rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))) / np.sqrt(2 * n)
    Z = np.linalg.qr(rng.standard_normal((m, m)))[0]
    Vd, Vx = _pack(Vc)
    t0 = time.perf_counter()
    with pytest.raises(B.JTRLanError) as ei:
        _rotate(Vd, n, m, Z, 2)
    assert ei.value.status == B.JTRLAN_ETIMEOUT
    assert 0.5 < time.perf_counter() - t0 < 60.0
    _check(_rotate(Vd, n, m, Z, 0), Vx, Z)
