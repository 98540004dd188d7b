"""The C ABI library loads, exports every symbol include/*.h declares, and its
host-side logic works without a GPU: argument checking (LAPACK's rule: the
return value is minus the 1-based position of the first illegal argument,
and nothing is launched) and the size-switch table.

Every call here either fails its argument check or is a quick return, so no
kernel is ever launched (the non-null pointers are placeholders that must
never reach a kernel).
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    from bfhelp import build_lib
    return build_lib()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(bf_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_symbols()
    for required in ("bf_dgemm", "bf_dgemm_strided_batched", "bf_dgemm_batched", "bf_dtrsm",
                     "bf_dpotrf", "bf_dpotrf_strided_batched", "bf_dpotrs", "bf_dgemm_vbatched",
                     "bf_dtrsm_vbatched", "bf_dpotrf_vbatched"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(so, n)]
    assert not missing, missing


NULL = None


def test_dgemm_illegal_arguments(lib):
    f = lib.bf_dgemm
    args = dict(ta=b"N", tb=b"N", m=4, n=4, k=4, alpha=1.0, A=1, lda=4, B=1, ldb=4, beta=0.0, C=1,
                ldc=4)

    def call(**kw):
        a = dict(args, **kw)
        return f(a["ta"], a["tb"], a["m"], a["n"], a["k"], a["alpha"], a["A"], a["lda"], a["B"],
                 a["ldb"], a["beta"], a["C"], a["ldc"], NULL)

    assert call(ta=b"X") == -1
    assert call(tb=b"?") == -2
    assert call(m=-1) == -3
    assert call(n=-1) == -4
    assert call(k=-2) == -5
    assert call(lda=3) == -8
    assert call(ta=b"T", lda=1, k=2) == -8  # op(A) = A^T: A has k rows
    assert call(ldb=3) == -10
    assert call(ldc=3) == -13
    assert call(A=NULL) == -7
    assert call(B=NULL) == -9
    assert call(C=NULL) == -12
    # quick returns launch nothing and succeed even without a GPU
    assert call(m=0) == 0
    assert call(n=0) == 0
    assert call(k=0, beta=1.0) == 0
    assert call(alpha=0.0, beta=1.0, A=NULL, B=NULL) == 0


def test_dgemm_strided_positions(lib):
    f = lib.bf_dgemm_strided_batched
    base = [b"N", b"T", 4, 4, 4, 1.0, 1, 4, 16, 1, 4, 16, 1.0, 1, 4, 16, 10, NULL]
    assert f(*base[:16], -1, NULL) == -17
    bad = list(base)
    bad[15] = 15  # strideC < ldc * n
    assert f(*bad) == -16
    bad = list(base)
    bad[10] = 3  # ldb < n for transb = 'T'
    assert f(*bad) == -11
    bad = list(base)
    bad[8] = -1
    assert f(*bad) == -9


def test_dtrsm_illegal_arguments(lib):
    f = lib.bf_dtrsm
    base = [b"R", b"L", b"T", b"U", 5, 3, 1.0, 1, 3, 1, 5, NULL]
    for pos, bad in ((0, b"X"), (1, b"Q"), (2, b"Z"), (3, b"A")):
        a = list(base)
        a[pos] = bad
        assert f(*a) == -(pos + 1)
    a = list(base)
    a[4] = -1
    assert f(*a) == -5
    a = list(base)
    a[8] = 2  # lda < n for side 'R'
    assert f(*a) == -9
    a = list(base)
    a[0] = b"L"  # side 'L': A is m x m, lda = 3 < m = 5
    assert f(*a) == -9
    a = list(base)
    a[10] = 4
    assert f(*a) == -11
    a = list(base)
    a[4] = 0
    assert f(*a) == 0


def test_dpotrf_and_dpotrs_arguments(lib):
    assert lib.bf_dpotrf(b"X", 4, 1, 4, NULL, NULL) == -1
    assert lib.bf_dpotrf(b"L", -1, 1, 4, NULL, NULL) == -2
    assert lib.bf_dpotrf(b"L", 4, NULL, 4, NULL, NULL) == -3
    assert lib.bf_dpotrf(b"L", 4, 1, 3, NULL, NULL) == -4
    assert lib.bf_dpotrf(b"U", 4, 1, 3, NULL, NULL) == -4  # uplo 'U' is checked like 'L'
    assert lib.bf_dpotrf(b"U", 0, NULL, 1, NULL, NULL) == 0   # n = 0: nothing launched
    assert lib.bf_dpotrf_strided_batched(b"L", 4, 1, 4, 15, NULL, 2, NULL) == -5
    assert lib.bf_dpotrf_strided_batched(b"L", 4, 1, 4, 16, NULL, -1, NULL) == -7
    assert lib.bf_dpotrf_strided_batched(b"L", 0, NULL, 1, 0, NULL, 5, NULL) == 0  # n = 0, no info
    assert lib.bf_dpotrs(b"L", 4, 2, 1, 4, 1, 3, NULL) == -7
    assert lib.bf_dpotrs(b"L", 4, -2, 1, 4, 1, 4, NULL) == -3
    assert lib.bf_dpotrs_strided_batched(b"L", 4, 2, 1, 4, 16, 1, 4, 7, 3, NULL) == -9


def test_status_strings(lib):
    assert lib.bf_status_string(0) == b"success"
    assert b"illegal" in lib.bf_status_string(-3)


def test_tune_table(lib):
    lib.tune_clear()
    try:
        default = lib.tune_query(lib.ROUTINE_DGEMM, 1, 24, 24, 24, 1000)
        assert default[1] == 24 and default[2] == 24  # whole 24 x 24 problem per super-tile
        lib.tune_set(lib.ROUTINE_DGEMM, 1, 16, 32, lib.VARIANT_DIRECT, 12, 24, 8, 2)
        got = lib.tune_query(lib.ROUTINE_DGEMM, 1, 24, 24, 24, 1000)
        # P = 2 of 18-thread super-tiles is raised to whole warps of at least 96 threads
        assert got == [lib.VARIANT_DIRECT, 12, 24, 8, 16]
        # other trans codes and sizes keep the default
        assert lib.tune_query(lib.ROUTINE_DGEMM, 0, 24, 24, 24, 1000) == default
        assert lib.tune_query(lib.ROUTINE_DGEMM, 1, 40, 40, 40, 1000)[1] == 40
        lib.tune_set(lib.ROUTINE_DPOTRF, 0, 1, 300, lib.VARIANT_BLOCKED, 128, 16)
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 0, 100, 100, 0, 10 ** 4)[:3] == [lib.VARIANT_BLOCKED, 128, 16]
        # dpotrf codes are the leading-dimension parity: an odd-lda entry leaves even lda alone
        lib.tune_set(lib.ROUTINE_DPOTRF, 1, 1, 300, lib.VARIANT_DIRECT, 64, 0, 8, 1)
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 100, 100, 0, 10 ** 5) == [lib.VARIANT_DIRECT, 64, 32, 8, 1]
        # a lane kernel needs tens of thousands of problems: small batches of orders 4..192 go
        # to the group form (p0 = 384 threads, p1 = 0: the group size from the launch's time
        # model), larger ones of n > 64 to the blocked sequence
        G6 = lib.VARIANT_GROUP
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 100, 100, 0, 10)[:3] == [G6, 384, 0]
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 0, 100, 100, 0, 10)[0] == G6
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 100, 100, 0, 10 ** 4)[0] == lib.VARIANT_BLOCKED
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 32, 32, 0, 1500)[:3] == [G6, 384, 0]
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 32, 32, 0, 10 ** 4)[:3] == [G6, 384, 0]
        # a forced group entry keeps its groups per SM (1..4); other values take the model
        lib.tune_set(lib.ROUTINE_DPOTRF, 1, 30, 34, G6 | lib.TUNE_FORCE, 512, 3)
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 32, 32, 0, 4096)[:3] == [G6, 512, 3]
        lib.tune_set(lib.ROUTINE_DPOTRF, 1, 30, 34, G6 | lib.TUNE_FORCE, 384, 9)
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 32, 32, 0, 4096)[:3] == [G6, 384, 0]
        lib.tune_clear()
        # past the group form's range, teams of 2 lanes per problem, then one problem per lane
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 48, 48, 0, 14000)[:4] == [lib.VARIANT_TEAM, 64, 32, 2]
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 48, 48, 0, 10 ** 5)[0] == lib.VARIANT_DIRECT
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 32, 32, 0, 24576)[0] == G6
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 32, 32, 0, 24577)[0] == lib.VARIANT_DIRECT
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 8, 8, 0, 4096)[0] == G6
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 0, 100, 100, 0, 4096)[0] != lib.VARIANT_TEAM
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 0, 200, 200, 0, 10)[0] == lib.VARIANT_CTA
        # the group form's measured bounds at large orders: up to 456 problems for orders
        # 112..143 (n = 128: 859 GFLOP/s against 688 with one problem per CTA), 304 from 144
        for code in (0, 1):
            assert lib.tune_query(lib.ROUTINE_DPOTRF, code, 128, 128, 0, 456)[0] == G6
            assert lib.tune_query(lib.ROUTINE_DPOTRF, code, 128, 128, 0, 532)[0] != G6
            assert lib.tune_query(lib.ROUTINE_DPOTRF, code, 144, 144, 0, 304)[0] == G6
            assert lib.tune_query(lib.ROUTINE_DPOTRF, code, 144, 144, 0, 384)[0] != G6
            assert lib.tune_query(lib.ROUTINE_DPOTRF, code, 193, 193, 0, 10)[0] != G6
        # a lane kernel on a small batch keeps two CTAs per SM: 13,000 problems -> 32 threads
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 8, 8, 0, 13000)[:2] == [lib.VARIANT_DIRECT, 32]
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 2, 2, 0, 10)[0] == lib.VARIANT_DIRECT
        # a forced entry holds at every batch size
        lib.tune_set(lib.ROUTINE_DPOTRF, 1, 90, 110, lib.VARIANT_DIRECT | lib.TUNE_FORCE, 64, 0, 8, 1)
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 100, 100, 0, 10) == [lib.VARIANT_DIRECT, 64, 32, 8, 1]
        with pytest.raises(lib.BFError):
            lib.tune_set(lib.ROUTINE_DPOTRF, 1, 90, 110, 7)
        # the team form: p2 is the team size (2 or 4; anything else is 4)
        lib.tune_set(lib.ROUTINE_DPOTRF, 0, 20, 30, lib.VARIANT_TEAM | lib.TUNE_FORCE, 128, 0, 2, 0)
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 0, 24, 24, 0, 10 ** 5)[:4] == [lib.VARIANT_TEAM, 128, 32, 2]
        lib.tune_set(lib.ROUTINE_DPOTRF, 0, 20, 30, lib.VARIANT_TEAM | lib.TUNE_FORCE, 128, 0, 3, 0)
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 0, 24, 24, 0, 10 ** 5)[3] == 4
        # dtrsm: fewer independent rows than the GPU needs -> the blocked form from order 64
        code_rltu = 8 + 2 + 1
        assert lib.tune_query(lib.ROUTINE_DTRSM, code_rltu, 256, 256, 0, 48)[0] == lib.VARIANT_BLOCKED
        assert lib.tune_query(lib.ROUTINE_DTRSM, code_rltu, 256, 256, 0, 2048)[0] != lib.VARIANT_BLOCKED
        assert lib.tune_query(lib.ROUTINE_DTRSM, code_rltu, 32, 32, 0, 10)[0] != lib.VARIANT_BLOCKED
        lib.tune_set(lib.ROUTINE_DTRSM, code_rltu, 1, 300, lib.VARIANT_DIRECT | lib.TUNE_FORCE, 8)
        assert lib.tune_query(lib.ROUTINE_DTRSM, code_rltu, 256, 256, 0, 48)[0] == lib.VARIANT_DIRECT
        # dgetrf: four lanes per problem from order 4 to 16; one problem per CTA above order 64 and
        # for small batches from order 17; the lane LU otherwise
        G = lib.ROUTINE_DGETRF
        assert lib.tune_query(G, 0, 128, 128, 0, 10 ** 6)[0] == lib.VARIANT_CTA
        assert lib.tune_query(G, 0, 32, 32, 0, 500)[0] == lib.VARIANT_CTA
        assert lib.tune_query(G, 0, 32, 32, 0, 10 ** 6)[0] == lib.VARIANT_DIRECT
        assert lib.tune_query(G, 0, 8, 8, 0, 10)[0] == lib.VARIANT_TEAM
        assert lib.tune_query(G, 0, 16, 16, 0, 10 ** 6)[0] == lib.VARIANT_TEAM
        assert lib.tune_query(G, 0, 4, 4, 0, 10 ** 6)[0] == lib.VARIANT_TEAM
        assert lib.tune_query(G, 0, 3, 3, 0, 10 ** 6)[0] == lib.VARIANT_DIRECT
        assert lib.tune_query(G, 0, 17, 17, 0, 10 ** 6)[0] == lib.VARIANT_DIRECT
        assert lib.tune_query(G, 0, 2000, 2000, 0, 10)[0] == lib.VARIANT_DIRECT  # the panel must fit
        lib.tune_set(G, 0, 1, 4000, lib.VARIANT_CTA | lib.TUNE_FORCE)
        assert lib.tune_query(G, 0, 8, 8, 0, 10 ** 6)[0] == lib.VARIANT_CTA
        assert lib.tune_query(G, 0, 2000, 2000, 0, 10)[0] == lib.VARIANT_DIRECT
        lib.tune_clear()
        lib.tune_set(G, 0, 1, 4000, lib.VARIANT_TEAM | lib.TUNE_FORCE)
        assert lib.tune_query(G, 0, 3, 3, 0, 10 ** 6)[0] == lib.VARIANT_TEAM
        assert lib.tune_query(G, 0, 17, 17, 0, 10)[0] == lib.VARIANT_DIRECT  # beyond the team form
        # defaults of the lane kernel: 8-row blocks for odd lda from n = 16, for even lda from n = 24
        lib.tune_clear()
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 0, 16, 16, 0, 10 ** 5)[3:] == [4, 2]
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 1, 16, 16, 0, 10 ** 5)[3:] == [8, 2]
        assert lib.tune_query(lib.ROUTINE_DPOTRF, 0, 24, 24, 0, 10 ** 5)[3:] == [8, 2]
        with pytest.raises(lib.BFError):
            lib.tune_set(7, 0, 1, 2, 0)
    finally:
        lib.reset_table()


def test_dsposv_and_backward_arguments(lib):
    f = lib.bf_dsposv_strided_batched
    W = lib.bf_dsposv_workspace_bytes(4, 1)
    assert W >= 4 * 4 * 4
    assert f(b"X", 4, 1, 1, 4, 16, 1, 4, 4, 1, 4, 4, None, None, 1e-12, 30, 256, W, 1, None) == -1
    assert f(b"L", 4, 1, 1, 3, 16, 1, 4, 4, 1, 4, 4, None, None, 1e-12, 30, 256, W, 1, None) == -5
    assert f(b"L", 4, 1, 1, 4, 16, 1, 4, 4, 1, 4, 4, None, None, -1.0, 30, 256, W, 1, None) == -15
    assert f(b"L", 4, 1, 1, 4, 16, 1, 4, 4, 1, 4, 4, None, None, 1e-12, 30, 256, W - 1, 1, None) == -18
    assert f(b"L", 4, 1, 1, 4, 16, 1, 4, 4, 1, 4, 4, None, None, 1e-12, 30, 8, W, 1, None) == -17
    assert f(b"L", 300, 1, 1, 300, 0, 1, 300, 0, 1, 300, 0, None, None, 1e-12, 30, 256,
             lib.bf_dsposv_workspace_bytes(300, 1), 1, None) == lib.ERR_NOT_SUPPORTED
    assert f(b"L", 0, 1, None, 1, 0, None, 1, 0, None, 1, 0, None, None, 1e-12, 30, None, 0, 1, None) == 0
    g = lib.bf_dpotrf_backward_strided_batched
    assert g(b"L", 4, 1, 3, 16, 1, 4, 16, 1, 4, 16, 1, None) == -4
    assert g(b"X", 4, 1, 4, 16, 1, 4, 16, 1, 4, 16, 1, None) == -1
    assert g(b"U", 4, 1, 4, 16, 1, 4, 16, 1, 4, 16, 0, None) == 0  # upper supported; empty batch
    h = lib.bf_dtrsm_backward_strided_batched
    assert h(b"R", b"L", b"T", b"N", 4, 4, 0.0, 1, 4, 16, 1, 4, 16, 1, 4, 16, None, 4, 0, 1, None) == -7
    k = lib.bf_dgemm_backward_strided_batched
    assert k(b"N", b"N", 4, 4, 4, 1.0, 1, 3, 16, 1, 4, 16, 1.0, 1, 4, 16, None, 4, 0, None, 4, 0, None, 4, 0,
             1, None) == -8
    # the dpotrs adjoint: (uplo, n, nrhs, L, ldl, sL, X, ldx, sX, Y, ldy, sY, XBbar, ldxb, sXB,
    # Lbar, ldlb, sLbar, batch, stream); every check returns before anything is launched
    d = lib.bf_dpotrs_backward_strided_batched

    def potrs_b(**kw):
        a = dict(uplo=b"L", n=4, nrhs=2, L=1, ldl=4, X=1, ldx=4, Y=1, ldy=4, Z=1, ldz=4, Lb=1, ldlb=4,
                 sLb=16, batch=2)
        a.update(kw)
        return d(a["uplo"], a["n"], a["nrhs"], a["L"], a["ldl"], 16, a["X"], a["ldx"], 8, a["Y"], a["ldy"], 8,
                 a["Z"], a["ldz"], 8, a["Lb"], a["ldlb"], a["sLb"], a["batch"], None)

    assert potrs_b(uplo=b"X") == -1
    assert potrs_b(n=-1) == -2
    assert potrs_b(nrhs=-1) == -3
    assert potrs_b(L=None) == -4
    assert potrs_b(ldl=3) == -5
    assert potrs_b(X=None) == -7
    assert potrs_b(ldx=3) == -8
    assert potrs_b(Y=None) == -10
    assert potrs_b(ldy=3) == -11
    assert potrs_b(Z=None) == -13
    assert potrs_b(ldz=3) == -14
    assert potrs_b(Lb=None) == -16
    assert potrs_b(ldlb=3) == -17
    assert potrs_b(sLb=15) == -18  # overlapping problems in Lbar
    assert potrs_b(batch=-1) == -19
    assert potrs_b(batch=0, L=None, X=None, Y=None, Z=None, Lb=None) == 0  # nothing to do
    assert potrs_b(n=0, L=None, X=None, Y=None, Z=None, Lb=None) == 0


def test_vbatched_illegal_call_arguments(lib):
    # the call's own arguments are checked on the host, nothing launched (no GPU needed); the
    # per-problem sizes live in device arrays and are checked by the kernels (dinfo)
    g = lib.bf_dgemm_vbatched
    ok = dict(ta=b"N", tb=b"T", m=1, n=1, k=1, A=1, lda=1, B=1, ldb=1, C=1, ldc=1, batch=3, mm=4, mn=4, mk=4)

    def gemm(**kw):
        a = dict(ok, **kw)
        return g(a["ta"], a["tb"], a["m"], a["n"], a["k"], 1.0, a["A"], a["lda"], a["B"], a["ldb"], 0.0,
                 a["C"], a["ldc"], a["batch"], a["mm"], a["mn"], a["mk"], NULL, NULL)
    assert gemm(ta=b"X") == -1
    assert gemm(tb=b"X") == -2
    assert gemm(batch=-1) == -14
    assert gemm(mm=-1) == -15
    assert gemm(mn=-1) == -16
    assert gemm(mk=-1) == -17
    assert gemm(batch=0, m=NULL) == 0
    for name, pos in (("m", -3), ("n", -4), ("k", -5), ("A", -7), ("lda", -8), ("B", -9), ("ldb", -10),
                      ("C", -12), ("ldc", -13)):
        assert gemm(**{name: NULL}) == pos
    t = lib.bf_dtrsm_vbatched

    def trsm(side=b"R", uplo=b"L", tr=b"T", diag=b"U", m=1, n=1, A=1, lda=1, B=1, ldb=1, batch=2, mm=3, mn=3):
        return t(side, uplo, tr, diag, m, n, 1.0, A, lda, B, ldb, batch, mm, mn, NULL, NULL)
    assert trsm(side=b"X") == -1
    assert trsm(uplo=b"X") == -2
    assert trsm(tr=b"X") == -3
    assert trsm(diag=b"X") == -4
    assert trsm(batch=-1) == -12
    assert trsm(mm=-1) == -13
    assert trsm(mn=-1) == -14
    assert trsm(m=NULL) == -5
    assert trsm(B=NULL) == -10
    p = lib.bf_dpotrf_vbatched
    assert p(b"X", 1, 1, 1, NULL, 1, 4, NULL) == -1
    assert p(b"L", 1, 1, 1, NULL, -1, 4, NULL) == -6
    assert p(b"L", 1, 1, 1, NULL, 1, -1, NULL) == -7
    assert p(b"U", 1, 1, 1, NULL, 0, 4, NULL) == 0  # upper is supported; an empty batch returns at once
    assert p(b"L", 1, 1, 1, NULL, 1, 1025, NULL) == lib.ERR_NOT_SUPPORTED
    assert p(b"L", NULL, 1, 1, NULL, 1, 4, NULL) == -2
    assert p(b"L", 1, 1, 1, NULL, 0, 4, NULL) == 0


def test_dpotrf_batch_switch_is_ordered(lib):
    """The built-in batch-size switch (no table entries): for every order, growing batches move
    from the group form to one problem per CTA, to teams of 4, then 2 lanes per problem, then one
    problem per lane (or, above order 64, the blocked sequence), and never back; the group form
    covers only orders 4..192, the team form only orders 12..64, and one problem per CTA only
    orders 16..256."""
    lib.tune_clear()
    try:
        stage = {lib.VARIANT_GROUP: -1, lib.VARIANT_CTA: 0, lib.VARIANT_TEAM: 1, lib.VARIANT_DIRECT: 3,
                 lib.VARIANT_BLOCKED: 3}
        batches = [1, 100, 600, 1000, 1500, 2000, 3000, 4096, 6144, 9728, 12288, 14592, 19456, 21000,
                   29127, 40000, 10 ** 5, 10 ** 6]
        for n in list(range(1, 70)) + [96, 128, 192, 256, 300]:
            for code in (0, 1):
                last = -1
                for b in batches:
                    v, T, _, p2, _ = lib.tune_query(lib.ROUTINE_DPOTRF, code, n, n, 0, b)
                    s = stage[v] + (1 if v == lib.VARIANT_TEAM and p2 == 2 else 0)
                    assert s >= last, (n, code, b)
                    last = s
                    if v == lib.VARIANT_TEAM:
                        assert 12 <= n <= 64 and p2 in (2, 4) and T == 64
                    if v == lib.VARIANT_CTA:
                        assert 16 <= n <= 256
                    if v == lib.VARIANT_GROUP:
                        assert 4 <= n <= 192 and T == 384
                        continue
                    assert T % 32 == 0 and 32 <= T <= 256
    finally:
        lib.tune_clear()


def test_batch_rules(lib, tmp_path):
    """bf_tune_set_batch_rule replaces the built-in batch bounds of dpotrf's small-batch forms
    for its order range and lda parity; the autotuner's table carries them (load_table)."""
    import json
    lib.tune_clear()
    try:
        q = lambda code, n, b: lib.tune_query(lib.ROUTINE_DPOTRF, code, n, n, 0, b)
        # the group form keeps its own bound (16,384 problems at n = 40..47); the rule decides
        # among the forms above it
        lib.tune_set_batch_rule(lib.ROUTINE_DPOTRF, -1, 40, 47, 17000, 18000, 20000)
        assert q(0, 44, 16384)[0] == lib.VARIANT_GROUP
        assert q(0, 44, 16385)[0] == lib.VARIANT_CTA
        assert q(0, 44, 17001)[:4] == [lib.VARIANT_TEAM, 64, 32, 4]
        assert q(1, 44, 20000)[:4] == [lib.VARIANT_TEAM, 64, 32, 2]
        assert q(0, 44, 20001)[0] == lib.VARIANT_DIRECT
        assert q(0, 48, 12288)[0] == lib.VARIANT_GROUP  # outside the rule: built-in bounds
        assert q(0, 48, 14000)[0] == lib.VARIANT_TEAM
        # only the lda-parity named; a negative cta bound keeps the built-in one (none at n = 44
        # above the group form's bound)
        lib.tune_set_batch_rule(lib.ROUTINE_DPOTRF, 1, 44, 44, -1, 0, -1)
        assert q(1, 44, 16385)[0] == lib.VARIANT_DIRECT  # team bounds (0, none): no team at all
        assert q(0, 44, 17001)[:4] == [lib.VARIANT_TEAM, 64, 32, 4]  # the even-lda rule above
        # a forced table entry is not affected
        lib.tune_set(lib.ROUTINE_DPOTRF, -1, 40, 47, lib.VARIANT_DIRECT | lib.TUNE_FORCE, 64, 0, 8, 2)
        assert q(0, 44, 50)[0] == lib.VARIANT_DIRECT
        lib.tune_clear()
        assert q(0, 44, 50)[0] == lib.VARIANT_GROUP and q(0, 44, 17001)[0] != lib.VARIANT_GROUP
        with pytest.raises(lib.BFError) as e:
            lib.tune_set_batch_rule(lib.ROUTINE_DGEMM, 0, 1, 2, 0, 0, 0)
        assert e.value.status == -1
        with pytest.raises(lib.BFError) as e:
            lib.tune_set_batch_rule(lib.ROUTINE_DPOTRF, 2, 1, 2, 0, 0, 0)
        assert e.value.status == -2
        with pytest.raises(lib.BFError) as e:
            lib.tune_set_batch_rule(lib.ROUTINE_DPOTRF, 0, 3, 2, 0, 0, 0)
        assert e.value.status == -3
        doc = {"entries": [], "batch_rules": [dict(routine=lib.ROUTINE_DPOTRF, code=-1, lo=40, hi=50,
                                                   cta_max=16400, team4_max=16500, team2_max=16600)]}
        path = tmp_path / "table.json"
        path.write_text(json.dumps(doc))
        assert lib.load_table(str(path)) == 0
        assert [q(0, 45, b)[0] for b in (16400, 16500, 16600, 16601)] == [
            lib.VARIANT_CTA, lib.VARIANT_TEAM, lib.VARIANT_TEAM, lib.VARIANT_DIRECT]
        assert q(0, 45, 100)[0] == lib.VARIANT_GROUP
    finally:
        lib.tune_clear()


def test_derive_batch_rule():
    """The autotuner's choice of batch bounds from measured times: the monotone schedule
    CTA -> team of 4 -> team of 2 -> table variant with the least summed time ratio."""
    from paper_1902_08115_gb300.autotune import derive_batch_rule
    best = {152: "cta", 304: "cta", 608: "team4", 1216: "team4", 2432: "team2", 4864: "table", 9728: "table"}
    rows = [(b, {f: (1.0 if f == w else 1.5) for f in ("cta", "team4", "team2", "table")}) for b, w in best.items()]
    assert derive_batch_rule(rows) == (304, 1216, 2432)
    # one noisy point out of order does not break the order: the least total loss wins
    rows[3] = (1216, {"cta": 1.0, "team4": 1.02, "team2": 1.5, "table": 1.5})
    assert derive_batch_rule(rows) == (304, 1216, 2432)
    # a form that cannot run at some order (no CTA form below order 16) is never scheduled
    rows = [(b, {"team4": 2.0, "team2": 1.0, "table": 1.2 if b < 1000 else 0.9}) for b in (152, 608, 2432)]
    assert derive_batch_rule(rows) == (0, 0, 608)
    # ties keep the table's variant
    rows = [(b, {"cta": 1.0, "team4": 1.0, "team2": 1.0, "table": 1.0}) for b in (152, 608)]
    assert derive_batch_rule(rows) == (0, 0, 0)


def test_dtrfill_illegal_arguments(lib):
    f = lib.bf_dtrfill_strided_batched
    assert f(b"X", 4, 1, 4, 16, NULL, 2, NULL) == -1
    assert f(b"L", -1, 1, 4, 16, NULL, 2, NULL) == -2
    assert f(b"L", 4, 1, 3, 16, NULL, 2, NULL) == -4
    assert f(b"L", 4, 1, 4, 15, NULL, 2, NULL) == -5
    assert f(b"L", 4, 1, 4, 16, NULL, -1, NULL) == -7
    assert f(b"L", 4, NULL, 4, 16, NULL, 2, NULL) == -3
    assert f(b"U", 0, NULL, 1, 0, NULL, 2, NULL) == 0
    assert f(b"L", 4, NULL, 4, 16, NULL, 0, NULL) == 0


def test_binding_refuses_mismatched_batch_counts(lib):
    """An operand holds one matrix per problem or one shared by all (batch count 1); any other
    count would make the kernels read past it, so the binding refuses before any launch."""
    import torch
    assert lib._bstride("A", 5, 16, 5) == 16
    assert lib._bstride("A", 1, 16, 5) == 0
    assert lib._bstride("A", 1, 16, 1) == 0
    with pytest.raises(ValueError, match="expected 5 or 1"):
        lib._bstride("A", 3, 16, 5)
    A = torch.zeros(3, 4, 4, dtype=torch.float64)
    C = torch.zeros(5, 4, 4, dtype=torch.float64)
    with pytest.raises(ValueError):
        lib.dgemm("N", "N", 1.0, A, C, 0.0, C)
    with pytest.raises(ValueError):
        lib.dtrsm("L", "L", "N", "N", 1.0, A, C)
    with pytest.raises(ValueError):
        lib.dpotrs(A, C)


def test_autograd_refuses_shared_operands(lib):
    """The adjoints write one gradient per problem; a batch-1 operand shared by every problem
    is refused up front (before the forward launches anything)."""
    import torch
    from paper_1902_08115_gb300.autograd import Gemm, TriSolve
    A1 = torch.zeros(1, 4, 4, dtype=torch.float64, requires_grad=True)
    B = torch.zeros(5, 4, 4, dtype=torch.float64, requires_grad=True)
    C = torch.zeros(5, 4, 4, dtype=torch.float64)
    with pytest.raises(ValueError, match="one matrix per problem"):
        Gemm.apply(A1, B, C, "N", "N", 1.0, 1.0, 4, 4, 4)
    with pytest.raises(ValueError, match="one matrix per problem"):
        TriSolve.apply(A1, B, "L", "L", "N", "N", 1.0, 4, 4)
