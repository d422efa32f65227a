"""GPU parity of the batched dense solver (one persistent launch over many instances of uneven order)
against the CPU FP64 oracle and brute-force dense diagonalisation, through the C ABI.

Tolerances: eigenvalues within 1e-10 relative of the oracle and of brute force (every eigenvalue of
a Hermitian J-symmetric matrix appears twice, so the wanted nev pairs are brute[0::2][:nev]); true
residuals ||A x - lambda x|| with unit x below the solve tolerance, recomputed here with the
oracle's matvec; X^H X = I and (J X*)^H X = O within 1e-10.
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


def _instances(sizes, seed0):
    return [inputs.dense_jsym(int(n) // 2, seed0 + i) for i, n in enumerate(sizes)]


def _batch(blocks, **kw):
    from paper_2001_07428_gb300.solver import JTRLanBatch
    return JTRLanBatch([a for a, _ in blocks], [b for _, b in blocks], device="cuda:0", **kw)


def _brute(A11, A12, nev, which):
    lam = np.linalg.eigvalsh(jsym.assemble_block_form(A11, A12))
    pairs = lam[0::2]
    assert np.allclose(lam[0::2], lam[1::2], rtol=0, atol=1e-9 * np.abs(lam).max())   # doubly degenerate
    return pairs[:nev] if which == "smallest" else pairs[::-1][:nev]


def _check_vectors(A11, A12, ev, X, tol):
    Xh = X.cpu().numpy()
    nev = len(ev)
    assert np.abs(Xh.conj().T @ Xh - np.eye(nev)).max() < 1e-10
    Y = np.stack([jsym.pair(Xh[:, i]) for i in range(nev)], axis=1)
    assert np.abs(Y.conj().T @ Xh).max() < 1e-10
    for i in range(nev):
        r = jsym.dense_matvec(A11, A12, Xh[:, i]) - ev[i] * Xh[:, i]
        assert np.linalg.norm(r) < tol, f"residual {i}: {np.linalg.norm(r):.3e}"


@pytest.mark.parametrize("precision", ["fp64", "mixed_reorth"])
def test_batch_small_matches_oracle(precision):
    # uneven orders, none a multiple of the 32-wide row chunks: several chunks and a ragged tail
    sizes = inputs.batched_dense_sizes(10, 64, 160, seed=5)
    blocks = _instances(sizes, 100)
    nev, m, mwin, tol = 8, 24, 12, 1e-10
    b = _batch(blocks, nev=nev, m=m, mwin=mwin, tol=tol, precision=precision)
    st = b.solve()
    assert st["n_ok"] == len(sizes) and st["graph"] == 1
    ev, res, ist = b.results()
    assert (ist[:, 2] == 0).all() and (res < tol).all()
    for i, (A11, A12) in enumerate(blocks):
        n = 2 * A11.shape[0]
        ref = tj.trlan_jsym(lambda x: jsym.dense_matvec(A11, A12, x), n, nev, m, mwin, 1e-12)
        rel = np.abs(ev[i] - ref["evals"]) / np.abs(ref["evals"])
        assert rel.max() < 1e-10, (i, n, rel.max())
        bf = _brute(A11, A12, nev, "smallest")
        assert (np.abs(ev[i] - bf) / np.abs(bf)).max() < 1e-10
        _check_vectors(A11, A12, ev[i], b.vectors(i), tol)
    b.close()


def test_batch_largest_matches_brute_force():
    sizes = [66, 98, 130, 64]
    blocks = _instances(sizes, 300)
    b = _batch(blocks, nev=6, m=20, mwin=10, tol=1e-10, which="largest")
    b.solve()
    ev, res, ist = b.results()
    for i, (A11, A12) in enumerate(blocks):
        bf = _brute(A11, A12, 6, "largest")
        assert (np.abs(ev[i] - bf) / np.abs(bf)).max() < 1e-10
        assert (np.diff(ev[i]) < 0).all()
        _check_vectors(A11, A12, ev[i], b.vectors(i), 1e-10)
    b.close()


def test_batch_single_instance_and_min_order():
    # count 1, and the smallest order the parameters allow (m < n/2)
    for n in (50, 256):
        blocks = _instances([n], 400 + n)
        b = _batch(blocks, nev=4, m=24, mwin=12, tol=1e-10)
        b.solve()
        ev, res, ist = b.results()
        bf = _brute(*blocks[0], 4, "smallest")
        assert (np.abs(ev[0] - bf) / np.abs(bf)).max() < 1e-10
        b.close()


def test_batch_replay_is_deterministic_and_shape_independent():
    sizes = inputs.batched_dense_sizes(40, 64, 200, seed=9)
    blocks = _instances(sizes, 500)
    b = _batch(blocks, nev=8, m=24, mwin=12, tol=1e-9)
    b.solve()
    ev1, res1, ist1 = b.results()
    b.solve()                                   # graph replay
    ev2, res2, ist2 = b.results()
    assert np.array_equal(ev1, ev2) and np.array_equal(ist1, ist2)
    b.set_shape(128, 1)                         # other CTA size: other reduction trees, same answers
    b.solve()
    ev3, _, ist3 = b.results()
    assert (ist3[:, 2] == 0).all()
    assert (np.abs(ev3 - ev1) / np.abs(ev1)).max() < 1e-11
    b.set_shape(512, 0)
    b.solve()
    ev4, _, _ = b.results()
    assert (np.abs(ev4 - ev1) / np.abs(ev1)).max() < 1e-11
    b.close()


def test_batch_not_converged_is_reported_per_instance():
    from paper_2001_07428_gb300 import binding as B
    blocks = _instances([128, 96], 700)
    b = _batch(blocks, nev=8, m=24, mwin=12, tol=1e-14, max_restarts=2)
    st = b.solve(check=False)
    assert st["status"] == B.JTRLAN_ENOCONV and st["n_ok"] == 0
    ev, res, ist = b.results()
    assert (ist[:, 2] == B.JTRLAN_ENOCONV).all() and (ist[:, 1] == 2).all()
    with pytest.raises(B.JTRLanError) as ei:
        b.vectors(0)
    assert ei.value.status == B.JTRLAN_ESTATE
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed_reorth"])
def test_batch_full_size_sampled(precision):
    """512 instances, n uniform over the even numbers 64..512, nev 8, m 24, residual 1e-8, in the
    autotuned launch shape and replayed from the CUDA graph, as the benchmark times it; sampled
    instances checked against brute force, every instance's status and residuals checked."""
    sizes = inputs.batched_dense_sizes(512, 64, 512, seed=2)
    blocks = _instances(sizes, 1000)
    tol = 1e-8
    b = _batch(blocks, nev=8, m=24, mwin=12, tol=tol, precision=precision)
    tuned = b.tune()
    assert tuned["threads"] in (128, 256, 512) and tuned["ctas_per_sm"] >= 1
    st = b.solve()
    assert st["n_ok"] == 512
    ev, res, ist = b.results()
    assert (ist[:, 2] == 0).all() and (res < tol).all()
    rng = np.random.default_rng(0)
    picks = {int(np.argmin(sizes)), int(np.argmax(sizes))} | set(rng.choice(512, 6, replace=False).tolist())
    for i in sorted(picks):
        A11, A12 = blocks[i]
        bf = _brute(A11, A12, 8, "smallest")
        assert (np.abs(ev[i] - bf) / np.abs(bf)).max() < 1e-10, (i, sizes[i])
        _check_vectors(A11, A12, ev[i], b.vectors(i), tol)
    b.close()


# ----------------------------------------------------------------------------- plain TRLAN (W removed)
@pytest.mark.parametrize("precision", ["fp64", "mixed_reorth"])
def test_plain_trlan_matches_oracle_on_case_a(precision):
    from paper_2001_07428_gb300.solver import JTRLan
    A11, A12, lam = inputs.case_a(400, 3)
    mv = lambda x: jsym.dense_matvec(A11, A12, x)
    top = np.sort(lam)[::-1][:5]
    s = JTRLan(kind="dense", A11=A11, A12=A12, nev=10, m=100, mwin=20, tol=1e-11, which="largest",
               precision=precision, plain_trlan=True, device="cuda:0")
    st = s.solve()
    ev, X, res = s.pairs()
    s.close()
    assert np.abs(ev - np.repeat(top, 2)).max() < 1e-12
    Xh = X.cpu().numpy()
    assert np.abs(Xh.conj().T @ Xh - np.eye(10)).max() < 1e-10
    for i in range(10):
        assert np.linalg.norm(mv(Xh[:, i]) - ev[i] * Xh[:, i]) < 1e-11
    ref = tj.trlan_jsym(mv, 400, 10, 100, 20, 1e-11, which="largest", use_w=False)
    js = JTRLan(kind="dense", A11=A11, A12=A12, nev=5, m=50, mwin=10, tol=1e-11, which="largest",
                precision=precision, device="cuda:0")
    st_js = js.solve()
    js.close()
    assert st["n_matvec"] > 1.5 * st_js["n_matvec"] and abs(st["n_matvec"] - ref["n_matvec"]) <= 0.2 * ref["n_matvec"]


@pytest.mark.parametrize("precision", ["fp64", "mixed_reorth"])
def test_batch_tile_shapes_agree_with_the_oracle(precision):
    """Every tile shape the autotuner searches (1 or 2 product rows per warp; all, 1, 2 or 4 update
    groups) returns the oracle's eigenvalues; the tuner's choice is readable afterwards."""
    sizes = inputs.batched_dense_sizes(12, 64, 300, seed=13)
    blocks = _instances(sizes, 900)
    nev, m, mwin, tol = 8, 24, 12, 1e-10
    ref = [tj.trlan_jsym(lambda x, a=a, b=b: jsym.dense_matvec(a, b, x), int(n), nev, m, mwin, 1e-12)["evals"]
           for (a, b), n in zip(blocks, sizes)]
    ref = np.array(ref)
    b = _batch(blocks, nev=nev, m=m, mwin=mwin, tol=tol, precision=precision)
    groups = (0, 1, 2, 4) if precision == "mixed_reorth" else (0,)
    for rows in (1, 2):
        for g in groups:
            b.set_tiles(rows, g)
            b.solve()
            ev, res, ist = b.results()
            assert (ist[:, 2] == 0).all() and (res < tol).all()
            assert (np.abs(ev - ref) / np.abs(ref)).max() < 1e-10, (rows, g)
    from paper_2001_07428_gb300 import binding as B
    tuned = B.jtrlan_batch_tune(b.b)
    assert tuned["mv_rows"] in (1, 2) and tuned["gs_groups"] in groups
    b.solve()
    ev, _, _ = b.results()
    assert (np.abs(ev - ref) / np.abs(ref)).max() < 1e-10
    b.close()
