"""GPU parity of the variable-size ("vbatched") dgemm, dtrsm, dpotrf and dpotrs against the oracle.

Each batch mixes problems of different sizes (zero sizes and padded leading dimensions
included); every problem is compared with the oracle run on that problem alone, normwise
relative error <= 1e-13.  Padding rows hold NaN and must come back untouched.  One problem
per batch carries an illegal argument (a leading dimension too small) and must be skipped
with dinfo = minus that argument's position, its matrices unchanged.
"""
import itertools

import numpy as np
import pytest
import torch

import bfsynth
from bfhelp import gpu, host, lower_part, normwise

pytestmark = pytest.mark.gpu

TOL = 1e-13


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from bfhelp import build_lib
    m = build_lib()
    m.reset_table()
    return m


def mat(rng, rows, cols, pad, fill=None):
    """Column-major (cols, ld) array: N(0,1) entries (or `fill`), NaN padding rows."""
    ld = max(rows, 1) + pad
    X = np.full((max(cols, 1), ld), np.nan)
    X[:cols, :rows] = rng.standard_normal((cols, rows)) if fill is None else fill
    return X


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (-0.5, 0.0), (0.0, 2.0), (1.5, -1.0)])
def test_dgemm_vbatched(bf, oracle, ta, tb, alpha, beta):
    rng = np.random.default_rng(11 + 3 * (ta == "T") + (tb == "T"))
    batch = 41
    ms = list(rng.integers(0, 37, batch))
    ns = list(rng.integers(0, 37, batch))
    ks = list(rng.integers(0, 37, batch))
    ms[0], ns[0], ks[0] = 5, 7, 0  # k = 0: C <= beta C
    ms[1], ns[1], ks[1] = 64, 70, 90  # more tiles than a CTA has threads
    As, Bs, Cs = [], [], []
    for q in range(batch):
        m, n, k = ms[q], ns[q], ks[q]
        ra, ca = (k, m) if ta == "T" else (m, k)
        rb, cb = (n, k) if tb == "T" else (k, n)
        As.append(mat(rng, ra, ca, q % 3))
        Bs.append(mat(rng, rb, cb, (q + 1) % 3))
        C = mat(rng, m, n, (q + 2) % 3)
        if beta == 0.0 and m and n:
            C[:n, :m] = np.nan  # beta == 0: C is not read
        Cs.append(C)
    bad = 7  # illegal: ldc < m (A and B legal)
    ms[bad], ns[bad], ks[bad] = 9, 4, 3
    As[bad] = mat(rng, *((3, 9) if ta == "T" else (9, 3)), 0)
    Bs[bad] = mat(rng, *((4, 3) if tb == "T" else (3, 4)), 0)
    Cs[bad] = mat(rng, 8, 4, 0)
    Cbad = Cs[bad].copy()
    Ag, Bg, Cg = [gpu(x) for x in As], [gpu(x) for x in Bs], [gpu(x) for x in Cs]
    dinfo = host(bf.dgemm_vbatched(ta, tb, alpha, Ag, Bg, beta, Cg, ms, ns, ks))
    assert dinfo[bad] == -13
    assert (np.delete(dinfo, bad) == 0).all()
    np.testing.assert_array_equal(host(Cg[bad]), Cbad)
    for q in range(batch):
        if q == bad:
            continue
        m, n, k = ms[q], ns[q], ks[q]
        out = host(Cg[q])
        if m == 0 or n == 0:
            np.testing.assert_array_equal(out, Cs[q])
            continue
        ref = oracle.dgemm(ta, tb, m, n, k, alpha, As[q], Bs[q], beta, np.nan_to_num(Cs[q], nan=0.0)
                           if beta == 0.0 else Cs[q])
        assert normwise(out[None, :n], ref[:, :n], m) <= TOL, q
        assert np.isnan(out[:n, m:]).all()


def tri(rng, order, pad, lower):
    """A well-conditioned triangular matrix (diagonal in [1, 2], off-diagonal entries of size
    1 / order), the other triangle NaN."""
    T = mat(rng, order, order, pad) * (0.5 / max(order, 1))
    for j in range(order):
        T[j, j] = 1.0 + rng.random()
        if lower:
            T[j, :j] = np.nan
        else:
            T[j, j + 1:order] = np.nan
    return T


@pytest.mark.parametrize("side,uplo,ta,diag", list(itertools.product("LR", "LU", "NT", "NU")))
def test_dtrsm_vbatched(bf, oracle, side, uplo, ta, diag):
    rng = np.random.default_rng(int.from_bytes((side + uplo + ta + diag).encode(), "little") % 1000)
    batch = 29
    ms = list(rng.integers(0, 33, batch))
    ns = list(rng.integers(0, 33, batch))
    ms[0], ns[0] = 40, 3
    As, Bs = [], []
    for q in range(batch):
        order = ms[q] if side == "L" else ns[q]
        As.append(tri(rng, order, q % 2, uplo == "L"))
        Bs.append(mat(rng, ms[q], ns[q], (q + 1) % 3))
    bad = 5  # illegal: lda < order of A
    ms[bad], ns[bad] = 6, 6
    As[bad] = tri(rng, 5, 0, uplo == "L")
    Bs[bad] = mat(rng, 6, 6, 0)
    Bbad = Bs[bad].copy()
    Ag, Bg = [gpu(x) for x in As], [gpu(x) for x in Bs]
    alpha = 0.75
    dinfo = host(bf.dtrsm_vbatched(side, uplo, ta, diag, alpha, Ag, Bg, ms, ns))
    assert dinfo[bad] == -9
    assert (np.delete(dinfo, bad) == 0).all()
    np.testing.assert_array_equal(host(Bg[bad]), Bbad)
    for q in range(batch):
        if q == bad:
            continue
        m, n = ms[q], ns[q]
        out = host(Bg[q])
        if m == 0 or n == 0:
            np.testing.assert_array_equal(out, Bs[q])
            continue
        ref = oracle.dtrsm(side, uplo, ta, diag, m, n, alpha, As[q], Bs[q])
        assert normwise(out[None, :n], ref[:, :n], m) <= TOL, q
        assert np.isnan(out[:n, m:]).all()


def spd(rng, n, pad):
    G = rng.standard_normal((n, n))
    S = np.full((max(n, 1), n + pad if n else 1 + pad), np.nan)
    if n:
        A = G @ G.T + n * np.eye(n)
        S[:n, :n] = A.T  # column-major
        for j in range(n):
            S[j, :j] = np.nan  # the strict upper triangle is not referenced
    return S


@pytest.mark.parametrize("uplo", "LU")
@pytest.mark.parametrize("nmax", [12, 32, 100, 300])
def test_dpotrf_vbatched(bf, oracle, nmax, uplo):
    rng = np.random.default_rng(nmax)
    batch = 23 if nmax <= 100 else 9
    ns = list(rng.integers(0, nmax + 1, batch))
    ns[0] = nmax
    As = [spd(rng, n, q % 3) for q, n in enumerate(ns)]
    fail = 3  # not positive definite at column 2
    ns[fail] = min(nmax, 6)
    As[fail] = spd(rng, ns[fail], 0)
    As[fail][1, 1] = -100.0
    bad = 4  # illegal: lda < n
    ns[bad] = min(nmax, 5)
    As[bad] = np.full((ns[bad], ns[bad] - 1), 1.0)
    if uplo == "U":  # the same matrices with the upper triangle stored, the strict lower one NaN
        for q, n in enumerate(ns):
            if q != bad:
                As[q][:n, :n] = As[q][:n, :n].T.copy()
    Abad = As[bad].copy()
    Ag = [gpu(x) for x in As]
    info = host(bf.dpotrf_vbatched(Ag, ns, uplo=uplo))
    assert info[bad] == -4
    np.testing.assert_array_equal(host(Ag[bad]), Abad)
    for q in range(batch):
        if q == bad:
            continue
        n = ns[q]
        out = host(Ag[q])
        if n == 0:
            assert info[q] == 0
            continue
        if uplo == "L":
            L, inf_o = oracle.dpotrf_l(np.nan_to_num(As[q], nan=0.0)[None], n)
            assert info[q] == inf_o[0], q
            if inf_o[0] == 0:
                assert normwise(lower_part(out[None], n), lower_part(L, n), n) <= TOL, q
            for j in range(n):
                assert np.isnan(out[j, :j]).all()  # upper triangle untouched
        else:
            U, inf_o = oracle.dpotrf_u(np.nan_to_num(As[q], nan=0.0)[None], n=n)
            assert info[q] == inf_o[0], q
            if inf_o[0] == 0:  # U^T in (ncols, ld) layout is lower: compare as lower parts
                ut = np.ascontiguousarray(np.transpose(out[None, :n, :n], (0, 2, 1)))
                ur = np.ascontiguousarray(np.transpose(U[:, :n, :n], (0, 2, 1)))
                assert normwise(lower_part(ut, n), lower_part(ur, n), n) <= TOL, q
            for j in range(n):
                assert np.isnan(out[j, j + 1:n]).all()  # strict lower triangle untouched
        assert np.isnan(out[:, n:]).all()


def test_vbatched_call_arguments(bf):
    z = torch.zeros(1, 1, dtype=torch.float64, device="cuda")
    with pytest.raises(bf.BFError) as e:
        bf.dpotrf_vbatched([z], [1025])
    assert e.value.status == bf.ERR_NOT_SUPPORTED
    with pytest.raises(bf.BFError) as e:
        bf.dpotrf_vbatched([z], [1], uplo="X")
    assert e.value.status == -1
    with pytest.raises(bf.BFError) as e:
        bf.dtrsm_vbatched("X", "L", "N", "N", 1.0, [z], [z], [1], [1])
    assert e.value.status == -1
    with pytest.raises(bf.BFError) as e:
        bf.dgemm_vbatched("N", "Q", 1.0, [z], [z], 0.0, [z], [1], [1], [1])
    assert e.value.status == -2


@pytest.mark.parametrize("uplo", "LU")
def test_dpotrs_vbatched_and_batched(bf, oracle, uplo):
    """Variable-size dpotrs (orders 0..70, 0..5 right-hand sides, padded leading dimensions) and
    the pointer-array dpotrs of a uniform batch, each against the oracle's dpotrs on the factor;
    an illegal problem is skipped with its dinfo and left untouched."""
    import ctypes
    rng = np.random.default_rng(77)
    batch = 25
    ns = [int(x) for x in rng.integers(0, 71, batch)]
    rs = [int(x) for x in rng.integers(0, 6, batch)]
    ns[0], rs[0] = 70, 5
    Ls, Bs, refs = [], [], []
    for q in range(batch):
        n, r = ns[q], rs[q]
        S = bfsynth.spd_batch(1, max(n, 1), max(n, 1) + q % 3, 900 + q).numpy()
        L, info = oracle.dpotrf_l(S, n)
        B = np.full((max(r, 1), max(n, 1) + (q + 1) % 2), np.nan)
        B[:r, :n] = rng.standard_normal((r, n))
        refs.append(oracle.dpotrs_l(L, B[None], n, r)[0] if n and r else B.copy())
        Lf = L[0]
        if uplo == "U":  # the same factor as U = L^T in the upper triangle
            Lf = Lf.copy()
            Lf[:n, :n] = Lf[:n, :n].T
        Ls.append(Lf)
        Bs.append(B)
    bad = 3
    ns[bad], rs[bad] = 4, 2
    Ls[bad] = np.ones((4, 3))  # lda 3 < n
    Bs[bad] = np.ones((2, 4))
    Lg, Bg = [gpu(x) for x in Ls], [gpu(x) for x in Bs]
    dinfo = host(bf.dpotrs_vbatched(Lg, Bg, ns, rs, uplo=uplo))
    assert dinfo[bad] == -5 and (np.delete(dinfo, bad) == 0).all()
    np.testing.assert_array_equal(host(Bg[bad]), Bs[bad])
    for q in range(batch):
        if q == bad or not (ns[q] and rs[q]):
            continue
        n, r = ns[q], rs[q]
        assert normwise(host(Bg[q])[None, :r, :n], refs[q][None, :r, :n], n) <= TOL, q
    # pointer-array dpotrs, uniform n = 19, 3 right-hand sides
    n, r, b = 19, 3, 6
    S = bfsynth.spd_batch(b, n, n + 1, 950).numpy()
    L, _ = oracle.dpotrf_l(S, n)
    B = bfsynth.randn_batch(b, n, r, n + 2, 951).numpy()
    ref = oracle.dpotrs_l(L, B, n, r)
    Lu = L.copy()
    if uplo == "U":
        for q in range(b):
            Lu[q, :n, :n] = L[q, :n, :n].T
    Lgs, Bgs = [gpu(Lu[q]) for q in range(b)], [gpu(B[q]) for q in range(b)]
    pa = torch.tensor([t.data_ptr() for t in Lgs], dtype=torch.int64, device="cuda")
    pb = torch.tensor([t.data_ptr() for t in Bgs], dtype=torch.int64, device="cuda")
    vp = ctypes.c_void_p
    assert bf.bf_dpotrs_batched(uplo.encode(), n, r, vp(pa.data_ptr()), n + 1, vp(pb.data_ptr()), n + 2, b,
                                bf._stream()) == 0
    got = np.stack([host(t) for t in Bgs])
    assert normwise(got, ref, n) <= TOL
