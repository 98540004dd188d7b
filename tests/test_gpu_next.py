"""GPU parity of dsyrk, the fused dsyrk + dpotrf, dtrmm, upper dpotrf / dpotrs and the
square-root Riccati recursion against the CPU oracle.

Every case runs the CUDA library through its C ABI (via the thin Python binding) on seeded
inputs and compares with the oracle on the same bytes.  Tolerance: normwise relative error
per problem <= 1e-13 for one routine call (the bar of the other FP64 tests); the Riccati
recursion chains 10 dependent stages of dtrmm + dsyrk + dpotrf, each within 1e-13, so its
factors are held to 1e-12.  Integer-valued inputs (dsyrk, dtrmm) must match bit for bit.
Sentinels: padding rows and the triangles a routine must not touch hold NaN and must come
back untouched.
"""
import itertools

import numpy as np
import pytest
import torch

import bfsynth
from bfhelp import forced, gpu, host, lower_part, normwise

pytestmark = pytest.mark.gpu

TOL = 1e-13
TOL_RICCATI = 1e-12


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from bfhelp import build_lib
    m = build_lib()
    m.reset_table()
    return m


def batch_for(n):
    return 3 if n >= 128 else (9 if n >= 48 else 37)


def tri_mask(n, uplo):
    """(ncols, ld) mask of the stored triangle of an n x n matrix."""
    M = np.tril(np.ones((n, n), bool)) if uplo == "L" else np.triu(np.ones((n, n), bool))
    return M.T  # element (i, j) lives at [j, i]


def rnd(shape, seed, integer=False):
    g = np.random.default_rng(seed)
    return g.integers(-3, 4, size=shape).astype(np.float64) if integer else g.standard_normal(shape)


# ----------------------------------------------------------------------------- dsyrk
@pytest.mark.parametrize("uplo,trans", list(itertools.product("LU", "NT")))
@pytest.mark.parametrize("n", [1, 3, 4, 5, 13, 24, 33, 64, 100, 130])
def test_dsyrk(bf, oracle, uplo, trans, n):
    k = max(1, (n * 2) // 3)
    batch = batch_for(n)
    rows, cols = (n, k) if trans == "N" else (k, n)
    A = np.full((batch, cols, rows + 2), np.nan)
    A[:, :, :rows] = rnd((batch, cols, rows), 10 + n)
    mask = tri_mask(n, uplo)
    C = np.full((batch, n, n + 3), np.nan)
    C[:, :, :n] = np.where(mask, rnd((batch, n, n), 20 + n), np.nan)  # other triangle: sentinel
    for alpha, beta in ((1.0, 1.0), (-0.5, 2.0), (1.0, 0.0), (2.0, 1.0)):
        Cin = C.copy()
        if beta == 0.0:
            Cin[:, :, :n] = np.nan  # beta = 0: C is not read
        ref = oracle.dsyrk(uplo, trans, n, k, alpha, A, beta, Cin)
        Cg = gpu(Cin)
        bf.dsyrk(uplo, trans, alpha, gpu(A), beta, Cg, n=n, k=k)
        out = host(Cg)
        got, want = np.where(mask, out[:, :, :n], 0.0), np.where(mask, ref[:, :, :n], 0.0)
        assert normwise(got, want, n) <= TOL, (alpha, beta)
        assert np.isnan(out[:, :, :n][:, ~mask]).all() and np.isnan(out[:, :, n:]).all()


@pytest.mark.parametrize("uplo,trans", list(itertools.product("LU", "NT")))
def test_dsyrk_integer_bit_exact_and_alpha_zero(bf, oracle, uplo, trans):
    n, k, batch = 21, 10, 5
    rows, cols = (n, k) if trans == "N" else (k, n)
    A = rnd((batch, cols, rows), 3, integer=True)
    C = rnd((batch, n, n), 4, integer=True)
    ref = oracle.dsyrk(uplo, trans, n, k, 1.0, A, 1.0, C)
    Cg = gpu(C)
    bf.dsyrk(uplo, trans, 1.0, gpu(A), 1.0, Cg, n=n, k=k)
    mask = tri_mask(n, uplo)
    np.testing.assert_array_equal(host(Cg)[:, mask], ref[:, mask])
    Cg = gpu(C)
    bf.dsyrk(uplo, trans, 0.0, gpu(np.full_like(A, np.nan)), 3.0, Cg, n=n, k=k)  # A not read
    np.testing.assert_array_equal(host(Cg)[:, mask], 3.0 * C[:, mask])


# ----------------------------------------------------------------------------- skinny dgemm
@pytest.mark.parametrize("variant", [0, 1], ids=["direct", "packed"])
@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_dgemm_rectangular_and_skinny(bf, oracle, variant, ta, tb):
    code = (2 if ta == "T" else 0) + (1 if tb == "T" else 0)
    for m, n, k in ((4, 256, 64), (256, 4, 64), (4, 4, 256), (128, 64, 4), (300, 4, 37), (1, 97, 5)):
        batch = 4
        rA, cA = (m, k) if ta == "N" else (k, m)
        rB, cB = (k, n) if tb == "N" else (n, k)
        A = np.full((batch, cA, rA + 1), np.nan)
        A[:, :, :rA] = rnd((batch, cA, rA), m + n + k)
        B = np.full((batch, cB, rB + 3), np.nan)
        B[:, :, :rB] = rnd((batch, cB, rB), m + n + k + 1)
        C = np.full((batch, n, m + 2), np.nan)
        C[:, :, :m] = rnd((batch, n, m), m + n + k + 2)
        ref = oracle.dgemm(ta, tb, m, n, k, -1.0, A, B, 1.0, C)
        Cg = gpu(C)
        with forced(bf, bf.ROUTINE_DGEMM, code, variant):
            bf.dgemm(ta, tb, -1.0, gpu(A), gpu(B), 1.0, Cg, m=m, n=n, k=k)
        out = host(Cg)
        assert normwise(out, ref, m) <= TOL, (m, n, k)
        assert np.isnan(out[:, :, m:]).all()


# ----------------------------------------------------------------------------- tiny problems
@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_dgemm_tiny(bf, oracle, ta, tb):
    code = (2 if ta == "T" else 0) + (1 if tb == "T" else 0)
    for (m, n, k) in ((4, 4, 4), (1, 1, 1), (3, 4, 2), (4, 1, 3), (2, 3, 4)):
        for pad in (0, 1):  # contiguous batches (16-byte staging) and padded ones (word staging)
            batch = 301
            rA, cA = (m, k) if ta == "N" else (k, m)
            rB, cB = (k, n) if tb == "N" else (n, k)
            A = np.full((batch, cA, rA + pad), np.nan)
            A[:, :, :rA] = rnd((batch, cA, rA), 600 + m + n + k, integer=True)
            B = np.full((batch, cB, rB + pad), np.nan)
            B[:, :, :rB] = rnd((batch, cB, rB), 601 + m + n + k, integer=True)
            C = np.full((batch, n, m + pad), np.nan)
            C[:, :, :m] = rnd((batch, n, m), 602 + m + n + k, integer=True)
            for alpha, beta in ((1.0, 1.0), (-1.0, 1.0), (2.0, 0.0), (0.5, -3.0)):
                Cin = C.copy()
                if beta == 0.0:
                    Cin[:, :, :m] = np.nan
                ref = oracle.dgemm(ta, tb, m, n, k, alpha, A, B, beta, Cin)
                Cg = gpu(Cin)
                with forced(bf, bf.ROUTINE_DGEMM, code, bf.VARIANT_TINY):
                    bf.dgemm(ta, tb, alpha, gpu(A), gpu(B), beta, Cg, m=m, n=n, k=k)
                out = host(Cg)
                np.testing.assert_array_equal(out[:, :, :m], ref[:, :, :m])  # integers: exact
                assert np.isnan(out[:, :, m:]).all()


@pytest.mark.parametrize("side,uplo,trans,diag", list(itertools.product("LR", "LU", "NT", "NU")))
def test_dtrsm_tiny(bf, oracle, side, uplo, trans, diag):
    code = (8 if side == "R" else 0) + (4 if uplo == "U" else 0) + (2 if trans == "T" else 0) + (1 if diag == "U" else 0)
    for m, n in ((1, 1), (4, 4), (3, 7), (8, 8), (8, 5)):
        for pad in (0, 1):
            k = m if side == "L" else n
            batch = 131
            A = np.full((batch, k, k + pad), np.nan)
            G = rnd((batch, k, k), 700 + m + n)
            A[:, :, :k] = 0.25 * G + 2.0 * np.eye(k)  # well-conditioned triangles, unit or not
            mask = tri_mask(k, uplo)
            A[:, :, :k] = np.where(mask, A[:, :, :k], np.nan)
            if diag == "U":
                for j in range(k):
                    A[:, j, j] = np.nan
            B = np.full((batch, n, m + pad), np.nan)
            B[:, :, :m] = rnd((batch, n, m), 800 + m + n)
            ref = oracle.dtrsm(side, uplo, trans, diag, m, n, 0.75, A, B)
            Bg = gpu(B)
            with forced(bf, bf.ROUTINE_DTRSM, code, bf.VARIANT_TINY):
                bf.dtrsm(side, uplo, trans, diag, 0.75, gpu(A), Bg, m=m, n=n)
            out = host(Bg)
            assert normwise(out, ref, m) <= TOL, (m, n, pad)
            assert np.isnan(out[:, :, m:]).all()


# ----------------------------------------------------------------------------- dsyrk + dpotrf
SP_VARIANTS = [("lane4", 0, 64, 0, 4, 2), ("lane8", 0, 64, 0, 8, 2), ("lane8u1", 0, 128, 0, 8, 1),
               ("blocked16", 2, 0, 16, 0, 0)]


@pytest.mark.parametrize("vname,variant,T,NB,R,U", SP_VARIANTS, ids=[v[0] for v in SP_VARIANTS])
@pytest.mark.parametrize("n", [1, 5, 12, 16, 24, 33, 48, 64, 96, 130])
def test_dsyrk_dpotrf(bf, oracle, vname, variant, T, NB, R, U, n):
    batch = batch_for(n)
    k = max(1, n // 2)
    for pad in (0, 3):
        A = np.full((batch, k, n + 1), np.nan)
        A[:, :, :n] = rnd((batch, k, n), 30 + n + pad)
        S = bfsynth.spd_batch(batch, n, n + pad, 40 + n + pad).numpy()
        for j in range(n):
            S[:, j, :j] = np.nan  # strict upper triangle: never read, never written
        F, info = oracle.dsyrk_dpotrf_l(n, k, A, S)
        assert (info == 0).all()
        Sg = gpu(S)
        with forced(bf, bf.ROUTINE_DPOTRF, -1, variant, T, NB, R, U):
            ig = bf.dsyrk_dpotrf(gpu(A), Sg, n=n, k=k)
        out = host(Sg)
        assert (host(ig) == 0).all()
        assert normwise(lower_part(out, n), lower_part(F, n), n) <= TOL
        for j in range(n):
            assert np.isnan(out[:, j, :j]).all()
        assert np.isnan(out[:, :, n:]).all()


def test_dsyrk_dpotrf_failures(bf, oracle):
    for n in (5, 40):
        batch, k = 7, 3
        A = rnd((batch, k, n), 50 + n)
        S = bfsynth.spd_batch(batch, n, n, 60 + n).numpy()
        S[2, 2, 2] = -1e3 * n  # problem 2 fails at column 3 despite the A A^T term
        S[5, n - 1, n - 1] = np.nan
        F, info = oracle.dsyrk_dpotrf_l(n, k, A, S)
        Sg = gpu(S)
        ig = host(bf.dsyrk_dpotrf(gpu(A), Sg, n=n, k=k))
        np.testing.assert_array_equal(ig, info)
        ok = info == 0
        assert normwise(lower_part(host(Sg)[ok], n), lower_part(F[ok], n), n) <= TOL


# ----------------------------------------------------------------------------- dtrmm
@pytest.mark.parametrize("side,uplo,trans,diag", list(itertools.product("LR", "LU", "NT", "NU")))
def test_dtrmm_all_cases(bf, oracle, side, uplo, trans, diag):
    for m, n in ((1, 1), (5, 3), (13, 17), (33, 24), (64, 40)):
        k = m if side == "L" else n
        batch = 11
        A = np.full((batch, k, k + 1), np.nan)
        A[:, :, :k] = rnd((batch, k, k), 70 + m + n)
        mask = tri_mask(k, uplo)
        A[:, :, :k] = np.where(mask, A[:, :, :k], np.nan)  # the other triangle is never read
        if diag == "U":
            for j in range(k):
                A[:, j, j] = np.nan  # nor the unit diagonal
        B = np.full((batch, n, m + 2), np.nan)
        B[:, :, :m] = rnd((batch, n, m), 80 + m + n)
        ref = oracle.dtrmm(side, uplo, trans, diag, m, n, 1.5, A, B)
        Bg = gpu(B)
        bf.dtrmm(side, uplo, trans, diag, 1.5, gpu(A), Bg, m=m, n=n)
        out = host(Bg)
        assert normwise(out, ref, m) <= TOL, (m, n)
        assert np.isnan(out[:, :, m:]).all()


@pytest.mark.parametrize("side", "LR")
def test_dtrmm_integer_bit_exact_and_alpha_zero(bf, oracle, side):
    m, n, batch = 19, 14, 6
    k = m if side == "L" else n
    A = rnd((batch, k, k), 90, integer=True)
    B = rnd((batch, n, m), 91, integer=True)
    for uplo, trans in itertools.product("LU", "NT"):
        ref = oracle.dtrmm(side, uplo, trans, "N", m, n, 1.0, A, B)
        Bg = gpu(B)
        bf.dtrmm(side, uplo, trans, "N", 1.0, gpu(A), Bg, m=m, n=n)
        np.testing.assert_array_equal(host(Bg), ref)
    Bg = gpu(B)
    bf.dtrmm(side, "L", "N", "N", 0.0, gpu(np.full_like(A, np.nan)), Bg, m=m, n=n)
    np.testing.assert_array_equal(host(Bg), np.zeros_like(B))


# ----------------------------------------------------------------------------- dpotrf / dpotrs upper
POTRF_U = [("direct4", 0, 64, 0, 4, 2), ("direct8", 0, 64, 0, 8, 2), ("packed", 1, 64, 0, 0, 0),
           ("blocked8", 2, 0, 8, 0, 0), ("blocked32", 2, 0, 32, 0, 0),
           ("cta", 4, 0, 0, 0, 0),
           ("team2", 5, 64, 0, 2, 0), ("team4", 5, 0, 0, 4, 0), ("group", 6, 0, 0, 0, 0)]


@pytest.mark.parametrize("vname,variant,T,NB,R,U", POTRF_U, ids=[v[0] for v in POTRF_U])
@pytest.mark.parametrize("n", [1, 3, 4, 7, 12, 16, 24, 33, 64, 100])
def test_dpotrf_upper(bf, oracle, vname, variant, T, NB, R, U, n):
    if variant == 1 and n > 16:
        pytest.skip("packed lane Cholesky holds whole problems in shared memory (small n)")
    batch = batch_for(n)
    for pad in (0, 3):
        S = bfsynth.spd_batch(batch, n, n + pad, 100 + n + pad).numpy()
        for j in range(n):
            S[:, j, j + 1:n] = np.nan  # strict lower triangle: never read, never written
        Uo, info = oracle.dpotrf_u(S, n=n)
        assert (info == 0).all()
        Sg = gpu(S)
        with forced(bf, bf.ROUTINE_DPOTRF, -1, variant, T, NB, R, U):
            ig = bf.dpotrf(Sg, n=n, uplo="U")
        out = host(Sg)
        assert (host(ig) == 0).all()
        up = tri_mask(n, "U")
        assert normwise(np.where(up, out[:, :, :n], 0), np.where(up, Uo[:, :, :n], 0), n) <= TOL
        for j in range(n):
            assert np.isnan(out[:, j, j + 1:n]).all()
        assert np.isnan(out[:, :, n:]).all()


def test_dpotrf_upper_failures_and_dpotrs(bf, oracle):
    n, batch = 30, 8
    S = bfsynth.spd_batch(batch, n, n, 123).numpy()
    S[3, 4, 4] = -50.0 * n
    Uo, info = oracle.dpotrf_u(S)
    Sg = gpu(S)
    np.testing.assert_array_equal(host(bf.dpotrf(Sg, uplo="U")), info)
    # solve with the upper factor: U^T U X = B
    good = np.nonzero(info == 0)[0]
    Sg = gpu(S[good].copy())
    bf.dpotrf(Sg, uplo="U")
    B = rnd((len(good), 3, n), 124)
    Xg = gpu(B)
    bf.dpotrs(Sg, Xg, n=n, nrhs=3, uplo="U")
    L, _ = oracle.dpotrf_l(np.ascontiguousarray(np.transpose(S[good], (0, 2, 1))))  # A symmetric: lower = upper^T
    Xo = oracle.dpotrs_l(L, B, n, 3)
    assert normwise(host(Xg), Xo, n) <= TOL


# ----------------------------------------------------------------------------- dgetrf / dgetrs
GETRF_VARIANTS = [("chosen", None), ("lane", 0), ("team", 5), ("cta", 4)]


@pytest.mark.parametrize("vname,variant", GETRF_VARIANTS, ids=[v[0] for v in GETRF_VARIANTS])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 13, 16, 17, 24, 33, 48, 64, 96, 130, 256, 384])
def test_dgetrf(bf, oracle, vname, variant, n):
    batch = batch_for(n)
    for pad in (0, 3):
        A = np.full((batch, n, n + pad), np.nan)
        A[:, :, :n] = rnd((batch, n, n), 200 + n + pad)
        LU, piv, info = oracle.dgetrf(A, m=n)
        Ag = gpu(A)
        if variant is None:
            pg, ig = bf.dgetrf(Ag, n=n)
        else:
            with forced(bf, bf.ROUTINE_DGETRF, 0, variant):
                pg, ig = bf.dgetrf(Ag, n=n)
        pg, ig, out = host(pg), host(ig), host(Ag)
        np.testing.assert_array_equal(ig, info)
        np.testing.assert_array_equal(pg, piv)  # same pivots: generic matrices have no near ties
        assert normwise(out, LU, n) <= TOL
        assert np.isnan(out[:, :, n:]).all()


@pytest.mark.parametrize("n", [4, 7, 16])
@pytest.mark.parametrize("batch", [1, 8, 17, 1000])
def test_dgetrf_team_tails_and_specials(bf, oracle, n, batch):
    """The four-lanes-per-problem LU (eight problems per warp, sixteen per CTA) on batches that
    leave a partial warp or CTA, with special problems planted: a NaN on a diagonal (kept as the
    pivot), a NaN below a diagonal (never taken), an infinity, ties of equal magnitude (the first
    row wins), a zero column (info) and an all-zero matrix.  Pivots and infos exactly as the
    oracle's; factors normwise against it where finite; and the same bits as the lane LU."""
    g = np.random.default_rng(900 + 10 * n + batch)
    pad = 3
    A = np.full((batch, n, n + pad), np.nan)
    A[:, :, :n] = g.standard_normal((batch, n, n))
    specials = []
    if batch >= 8:
        A[1, 0, 0] = np.nan                      # NaN on the diagonal: row 0 stays the pivot
        A[2, 2, 1] = np.nan                      # NaN below a diagonal: never the pivot
        A[3, 1, 3] = np.inf                      # an infinity
        A[4, :, 0] = 1.0                         # equal magnitudes: the first row wins
        A[4, 2, 0] = -1.0
        A[5, :, 2] = 0.0                         # a zero column -> info 3
        A[6, :, :n] = 0.0                        # all zero -> info 1
        specials = [1, 2, 3, 4, 5, 6]
    LU, piv, info = oracle.dgetrf(A, m=n)
    outs = {}
    for name, v in (("team", bf.VARIANT_TEAM), ("lane", bf.VARIANT_DIRECT)):
        Ag = gpu(A)
        with forced(bf, bf.ROUTINE_DGETRF, 0, v):
            pg, ig = bf.dgetrf(Ag, n=n)
        outs[name] = (host(Ag), host(pg), host(ig))
    out, pg, ig = outs["team"]
    np.testing.assert_array_equal(ig, info)
    np.testing.assert_array_equal(pg, piv)
    finite = np.isfinite(LU).all(axis=(1, 2)) & np.isfinite(out[:, :, :n]).all(axis=(1, 2))
    finite &= ~np.isin(np.arange(batch), specials)
    assert normwise(out[finite], LU[finite], n) <= TOL
    assert np.isnan(out[:, :, n:]).all()                      # padding untouched
    for a, b in zip(outs["team"], outs["lane"]):
        np.testing.assert_array_equal(a, b)                    # same bits (NaN where NaN)


@pytest.mark.parametrize("vname,variant", GETRF_VARIANTS, ids=[v[0] for v in GETRF_VARIANTS])
@pytest.mark.parametrize("n", [9, 40])
def test_dgetrf_singular_and_permutation(bf, oracle, vname, variant, n):
    batch = 4
    A = rnd((batch, n, n), 300)
    A[1, 4, :] = 0.0                               # problem 1: column 4 zero -> info 5
    A[2] = np.eye(n)[np.random.default_rng(1).permutation(n)]  # problem 2: a permutation matrix
    A[3, :, :] = 0.0                               # problem 3: all zero -> info 1
    A[0, n - 3, :] = 0.0                           # problem 0: zero column in the last panel
    LU, piv, info = oracle.dgetrf(A, m=n)
    Ag = gpu(A)
    if variant is None:
        pg, ig = bf.dgetrf(Ag)
    else:
        with forced(bf, bf.ROUTINE_DGETRF, 0, variant):
            pg, ig = bf.dgetrf(Ag)
    np.testing.assert_array_equal(host(ig), info)
    assert info[1] == 5 and info[3] == 1 and info[2] == 0 and info[0] == n - 2
    np.testing.assert_array_equal(host(pg), piv)
    np.testing.assert_array_equal(host(Ag)[2], LU[2])  # integer-exact: no rounding happens


@pytest.mark.parametrize("m,n", [(7, 3), (3, 7), (33, 17), (17, 33), (1, 5), (5, 1), (100, 20), (20, 100),
                                 (300, 64), (64, 300), (384, 40), (1024, 16)])
def test_dgetrf_rectangular(bf, oracle, m, n):
    """m x n LU (one problem per CTA): pivots identical to the oracle's, factors within the
    tolerance, padding rows untouched; failures (a zero column) reported as the oracle does."""
    batch = 5
    A = np.full((batch, n, m + 3), np.nan)
    A[:, :, :m] = rnd((batch, n, m), 600 + m + n)
    A[2, min(n, m) // 2, :m] = 0.0  # problem 2: a zero column inside the factored part
    LU, piv, info = oracle.dgetrf(A, m=m, n=n)
    Ag = gpu(A)
    pg, ig = bf.dgetrf(Ag, m=m, n=n)
    pg, ig, out = host(pg), host(ig), host(Ag)
    assert pg.shape == (batch, min(m, n))
    np.testing.assert_array_equal(ig, info)
    assert info[2] == min(n, m) // 2 + 1
    np.testing.assert_array_equal(pg, piv)
    ok = info == 0
    assert normwise(out[ok], LU[ok], m) <= TOL
    assert np.isnan(out[:, :, m:]).all()


@pytest.mark.parametrize("trans", "NT")
@pytest.mark.parametrize("n", [1, 7, 32, 65])
def test_dgetrs(bf, oracle, trans, n):
    batch, r = 9, 3
    A = rnd((batch, n, n), 400 + n) + 2 * np.eye(n)
    B = np.full((batch, r, n + 1), np.nan)
    B[:, :, :n] = rnd((batch, r, n), 500 + n)
    LU, piv, info = oracle.dgetrf(A, m=n)
    Xo = oracle.dgetrs(trans, LU, piv, B, n, r)
    Ag = gpu(A)
    pg, _ = bf.dgetrf(Ag)
    Bg = gpu(B)
    bf.dgetrs(trans, Ag, pg, Bg, n=n, nrhs=r)
    out = host(Bg)
    assert normwise(out, Xo, n) <= TOL
    assert np.isnan(out[:, :, n:]).all()


# ----------------------------------------------------------------------------- Riccati
def riccati_inputs(batch, N, nx, nu, seed):
    g = np.random.default_rng(seed)
    m = nx + nu
    A = g.standard_normal((batch, N, nx, nx)) / np.sqrt(nx)
    B = g.standard_normal((batch, N, nx, nu)) / np.sqrt(nx)
    G = g.standard_normal((batch, N, m, m))
    RSQ = G @ np.swapaxes(G, -1, -2) + m * np.eye(m)
    H = g.standard_normal((batch, nx, nx))
    QN = H @ np.swapaxes(H, -1, -2) + nx * np.eye(nx)
    BAt = np.concatenate([np.swapaxes(B, -1, -2), np.swapaxes(A, -1, -2)], axis=-2)  # (batch, N, m, nx)
    # column-major (ncols, ld) layouts
    return (np.ascontiguousarray(np.swapaxes(BAt, -1, -2)), np.ascontiguousarray(np.swapaxes(RSQ, -1, -2)),
            np.ascontiguousarray(np.swapaxes(QN, -1, -2)))


@pytest.mark.parametrize("fused", [True, False], ids=["fused", "blas"])
@pytest.mark.parametrize("nx,nu", [(8, 4), (24, 12), (40, 20)])
def test_riccati(bf, oracle, fused, nx, nu):
    N, batch = 10, 24
    BAt, RSQ, QN = riccati_inputs(batch, N, nx, nu, 7 * nx + nu)
    Fo, info_o = oracle.riccati(BAt, RSQ, QN, nx, nu)
    assert (info_o == 0).all()
    Fg, ig = bf.riccati(gpu(BAt), gpu(RSQ), gpu(QN), nx, nu, fused=fused)
    Fg, ig = host(Fg), host(ig)
    assert (ig == 0).all()
    m = nx + nu
    for s in range(N + 1):
        size = nx if s == N else m
        got, want = lower_part(Fg[:, s], size), lower_part(Fo[:, s], size)
        assert normwise(got, want, size) <= TOL_RICCATI, s


def test_riccati_failure_stage(bf, oracle):
    N, nx, nu, batch = 6, 8, 4, 5
    BAt, RSQ, QN = riccati_inputs(batch, N, nx, nu, 99)
    RSQ[2, 3, 1, 1] = -1e4  # problem 2 fails at stage 3, column 2
    QN[4, 0, 0] = -1.0      # problem 4 fails in the terminal factorisation, column 1
    Fo, info_o = oracle.riccati(BAt, RSQ, QN, nx, nu)
    assert info_o[2] == 3002 and info_o[4] == 1000 * N + 1
    for fused in (True, False):
        _, ig = bf.riccati(gpu(BAt), gpu(RSQ), gpu(QN), nx, nu, fused=fused)
        np.testing.assert_array_equal(host(ig), info_o)
