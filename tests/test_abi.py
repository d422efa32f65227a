"""Host-side checks of the C ABI that need no GPU: the library builds and loads, exports every
function include/jtrlan.h declares, the ctypes structs match the C layout, and invalid arguments
are rejected before any CUDA work."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2001_07428_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "jtrlan.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB_PATH):
        from paper_2001_07428_gb300 import build
        build.build()
    return B.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(jtrlan_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_abi():
    assert {"jtrlan_create", "jtrlan_apply", "jtrlan_solve", "jtrlan_pairs"} <= set(declared_functions())


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (jtrlan_\w+)", out))
    assert set(declared_functions()) <= exported


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "jtrlan.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(jtrlan_operator), offsetof(jtrlan_operator, n),
         offsetof(jtrlan_operator, m0), offsetof(jtrlan_operator, a11), offsetof(jtrlan_operator, W));
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(jtrlan_params), offsetof(jtrlan_params, tol),
         offsetof(jtrlan_params, v1), offsetof(jtrlan_params, check_jsym), offsetof(jtrlan_params, profile),
         offsetof(jtrlan_params, filter_hi), offsetof(jtrlan_params, filter_final_coeffs),
         offsetof(jtrlan_params, plain_trlan), offsetof(jtrlan_params, rotate_simt),
         offsetof(jtrlan_params, invert), offsetof(jtrlan_params, cg_tol), offsetof(jtrlan_params, cg_max_iter),
         offsetof(jtrlan_params, gs_split));
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(jtrlan_stats), offsetof(jtrlan_stats, n_restarts),
         offsetof(jtrlan_stats, solve_ms), offsetof(jtrlan_stats, n_launches), offsetof(jtrlan_stats, n_ritz_fallbacks),
         offsetof(jtrlan_stats, n_matvec_fp32), offsetof(jtrlan_stats, n_matvec_inner),
         offsetof(jtrlan_stats, n_cg_iters));
  printf("%zu %zu %zu %zu\n", sizeof(jtrlan_profile), offsetof(jtrlan_profile, ms),
         offsetof(jtrlan_profile, launches), offsetof(jtrlan_profile, work));
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(jtrlan_batch_stats), offsetof(jtrlan_batch_stats, n_matvec),
         offsetof(jtrlan_batch_stats, max_restarts), offsetof(jtrlan_batch_stats, graph),
         offsetof(jtrlan_batch_stats, solve_ms), offsetof(jtrlan_batch_stats, phase_frac));
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [list(map(int, l.split())) for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines()]
    O, P, S, F = B.jtrlan_operator, B.jtrlan_params, B.jtrlan_stats, B.jtrlan_profile
    assert got[0] == [ctypes.sizeof(O), O.n.offset, O.m0.offset, O.a11.offset, O.W.offset]
    assert got[1] == [ctypes.sizeof(P), P.tol.offset, P.v1.offset, P.check_jsym.offset, P.profile.offset,
                      P.filter_hi.offset, P.filter_final_coeffs.offset, P.plain_trlan.offset,
                      P.rotate_simt.offset, P.invert.offset, P.cg_tol.offset, P.cg_max_iter.offset,
                      P.gs_split.offset]
    assert got[2] == [ctypes.sizeof(S), S.n_restarts.offset, S.solve_ms.offset, S.n_launches.offset,
                      S.n_ritz_fallbacks.offset, S.n_matvec_fp32.offset, S.n_matvec_inner.offset,
                      S.n_cg_iters.offset]
    assert got[3] == [ctypes.sizeof(F), F.ms.offset, F.launches.offset, F.work.offset]
    Q = B.jtrlan_batch_stats
    assert got[4] == [ctypes.sizeof(Q), Q.n_matvec.offset, Q.max_restarts.offset, Q.graph.offset,
                      Q.solve_ms.offset, Q.phase_frac.offset]


def test_status_strings(lib):
    for s in range(9):
        assert lib.jtrlan_status_string(s)


DUMMY = 0x1000  # never dereferenced: validation fails before any copy


@pytest.mark.parametrize("case", ["odd_n", "stencil_n", "nev_ge_m", "m_ge_half", "neg_mwin", "tol",
                                  "which", "null_links", "kind", "precision", "big_m"])
def test_invalid_arguments_rejected_without_gpu(lib, case):
    op = B.stencil_operator((4, 4, 4, 4), 8.5, 0.3, DUMMY, DUMMY)
    prm = B.params(6, 24, 12, 1e-10)
    if case == "odd_n":
        op = B.dense_operator(201, DUMMY, DUMMY)
    elif case == "stencil_n":
        op.n = op.n + 2
    elif case == "nev_ge_m":
        prm.nev = 24
    elif case == "m_ge_half":
        prm.m = op.n // 2
    elif case == "neg_mwin":
        prm.mwin = -1
    elif case == "tol":
        prm.tol = 0.0
    elif case == "which":
        prm.which = 7
    elif case == "null_links":
        op.U = None
    elif case == "kind":
        op.kind = 9
    elif case == "precision":
        prm.precision = 5
    elif case == "big_m":
        op = B.dense_operator(4000, DUMMY, DUMMY)
        prm.m = 1024
    with pytest.raises(B.JTRLanError) as ei:
        B.jtrlan_create(op, prm, 0)
    assert ei.value.status == B.JTRLAN_EINVAL


def test_null_context_calls(lib):
    assert lib.jtrlan_solve(None, None) == B.JTRLAN_EINVAL
    assert lib.jtrlan_pairs(None, 0, None, None, None) == B.JTRLAN_EINVAL
    assert lib.jtrlan_apply(None, None, None) == B.JTRLAN_EINVAL
    assert lib.jtrlan_apply_filter(None, None, None) == B.JTRLAN_EINVAL
    assert lib.jtrlan_get_profile(None, None) == B.JTRLAN_EINVAL
    lib.jtrlan_destroy(None)


@pytest.mark.parametrize("case", ["count", "stencil", "odd_n", "m_ge_half", "big_m", "big_nev", "mixed", "v1",
                                  "check_jsym", "which", "tol"])
def test_batch_invalid_arguments_rejected_without_gpu(lib, case):
    ops = [B.dense_operator(n, DUMMY, DUMMY) for n in (64, 100, 128)]
    prm = B.params(8, 24, 12, 1e-8)
    if case == "count":
        ops = []
    elif case == "stencil":
        ops[1] = B.stencil_operator((4, 4, 4, 4), 8.5, 0.3, DUMMY, DUMMY)
    elif case == "odd_n":
        ops[2].n = 129
    elif case == "m_ge_half":
        ops[0].n = 48
    elif case == "big_m":
        ops = [B.dense_operator(400, DUMMY, DUMMY)]
        prm.m = 65
    elif case == "big_nev":
        ops = [B.dense_operator(400, DUMMY, DUMMY)]
        prm.m, prm.nev = 60, 33
    elif case == "mixed":
        prm.precision = B.JTRLAN_MIXED
    elif case == "v1":
        prm.v1 = DUMMY
    elif case == "check_jsym":
        prm.check_jsym = 1
    elif case == "which":
        prm.which = 3
    elif case == "tol":
        prm.tol = -1.0
    if case == "count":
        b = ctypes.c_void_p()
        st = lib.jtrlan_batch_create(0, None, ctypes.byref(prm), None, ctypes.byref(b))
        assert st == B.JTRLAN_EINVAL and not b.value
        return
    with pytest.raises(B.JTRLanError) as ei:
        B.jtrlan_batch_create(ops, prm, 0)
    assert ei.value.status == B.JTRLAN_EINVAL


def test_batch_null_calls(lib):
    assert lib.jtrlan_batch_solve(None, None) == B.JTRLAN_EINVAL
    assert lib.jtrlan_batch_results(None, None, None, None) == B.JTRLAN_EINVAL
    assert lib.jtrlan_batch_vectors(None, 0, None) == B.JTRLAN_EINVAL
    assert lib.jtrlan_batch_tune(None, None, None, None) == B.JTRLAN_EINVAL
    assert lib.jtrlan_batch_set_shape(None, 256, 0) == B.JTRLAN_EINVAL
    lib.jtrlan_batch_destroy(None)


def test_rotate_df_rejects_bad_arguments_before_touching_the_device(lib):
    # every check below fails on the host, so the dummy (never dereferenced) pointers are safe
    d = ctypes.c_void_p(16)
    assert lib.jtrlan_rotate_df(None, 10, 4, d, 2, d, 0, None) == B.JTRLAN_EINVAL
    assert lib.jtrlan_rotate_df(d, 0, 4, d, 2, d, 0, None) == B.JTRLAN_EINVAL
    assert lib.jtrlan_rotate_df(d, 10, 0, d, 2, d, 0, None) == B.JTRLAN_EINVAL
    assert lib.jtrlan_rotate_df(d, 10, 4, d, 0, d, 0, None) == B.JTRLAN_EINVAL
    assert lib.jtrlan_rotate_df(d, 10, 4, d, 2, d, 3, None) == B.JTRLAN_EINVAL
    assert lib.jtrlan_rotate_df(d, 10, 321, d, 2, d, 2, None) == B.JTRLAN_EINVAL
    assert lib.jtrlan_rotate_df(d, 10, 321, d, 2, d, 0, None) == B.JTRLAN_EINVAL   # tensor cores: m <= 320
    assert "320" in lib.jtrlan_last_error().decode()


def test_invert_mode_parameter_checks(lib):
    # invert mode needs FP64, the smallest end and no filter; all rejected before any device work
    import numpy as np
    n = 12
    a = ctypes.c_void_p(16)
    op = B.dense_operator(n, a, a)
    for kw in (dict(precision=B.JTRLAN_MIXED_REORTH), dict(which=B.JTRLAN_LARGEST), dict(cg_tol=-1.0),
               dict(cg_max_iter=-3)):
        args = dict(which=B.JTRLAN_SMALLEST, precision=B.JTRLAN_FP64)
        args.update(kw)
        prm = B.params(2, 4, 1, 1e-8, invert=1, **args)
        with pytest.raises(B.JTRLanError) as ei:
            B.jtrlan_create(op, prm, 0)
        assert ei.value.status == B.JTRLAN_EINVAL
    prm = B.params(2, 4, 1, 1e-8, invert=1, filter_final_coeffs=np.ones(3), filter_window=(0.0, 1.0))
    prm.filter_final_degree = 2
    with pytest.raises(B.JTRLanError) as ei:
        B.jtrlan_create(op, prm, 0)
    assert ei.value.status == B.JTRLAN_EINVAL
