"""GPU parity of dgemm / dtrsm / dpotrf / dpotrs against the CPU oracle.

Every case runs the CUDA library through its C ABI (via the thin Python
binding) on seeded inputs and compares element by element with the oracle
on the same bytes.  Tolerance: normwise relative error per problem <= 1e-13
for the FP64 paths; integer-valued inputs must match bit for bit.  Every
kernel variant of the size switch is forced in turn through the tuning
table, so the direct, packed and blocked forms are each checked.
Sentinels: leading-dimension padding rows and unused triangles hold NaN and
must come back untouched (and must not leak into results).
"""
import itertools

import numpy as np
import pytest
import torch

import bfsynth
from bfhelp import forced, gpu, host, lower_part, normwise

pytestmark = pytest.mark.gpu

TOL = 1e-13
TRANS = list(itertools.product("NT", "NT"))
SMALL_N = [1, 2, 3, 4, 5, 7, 8, 12, 13, 16, 24, 31, 32, 48, 64, 67, 96, 128, 130, 192, 256]


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from bfhelp import build_lib
    m = build_lib()
    m.reset_table()
    return m


def small_batch(n):
    return 3 if n >= 128 else (9 if n >= 48 else 37)


def code2(ta, tb):
    return (2 if ta == "T" else 0) + (1 if tb == "T" else 0)


# ----------------------------------------------------------------------------- dgemm
@pytest.mark.parametrize("variant", [0, 1], ids=["direct", "packed"])
@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("n", SMALL_N)
def test_dgemm_square(bf, oracle, variant, ta, tb, n):
    for pad in (0, 3):
        batch = small_batch(n)
        ld = n + pad
        seed = 1000 * n + 10 * pad + code2(ta, tb)
        A = bfsynth.randn_batch(batch, n, n, ld, seed).numpy()
        B = bfsynth.randn_batch(batch, n, n, ld, seed + 1).numpy()
        C = bfsynth.randn_batch(batch, n, n, ld, seed + 2).numpy()
        ref = oracle.dgemm(ta, tb, n, n, n, 1.0, A, B, 1.0, C)
        Cg = gpu(C)
        with forced(bf, bf.ROUTINE_DGEMM, code2(ta, tb), variant):
            bf.dgemm(ta, tb, 1.0, gpu(A), gpu(B), 1.0, Cg, m=n, n=n, k=n)
        out = host(Cg)
        assert normwise(out, ref, n) <= TOL
        assert np.isnan(out[:, :, n:]).all()


@pytest.mark.parametrize("variant", [0, 1], ids=["direct", "packed"])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-1.0, 1.0), (0.5, -2.0), (2.0, 0.0), (1.0, 3.0),
                                        (0.0, 0.5), (0.0, 0.0)])
def test_dgemm_scalars(bf, oracle, variant, alpha, beta):
    for (m, n, k) in [(5, 7, 3), (24, 24, 24), (67, 33, 90)]:
        for ta, tb in TRANS:
            batch = 5
            rA, cA = (m, k) if ta == "N" else (k, m)
            rB, cB = (k, n) if tb == "N" else (n, k)
            A = bfsynth.randn_batch(batch, rA, cA, rA + 1, 7).numpy()
            B = bfsynth.randn_batch(batch, rB, cB, rB + 2, 8).numpy()
            C = bfsynth.randn_batch(batch, m, n, m + 1, 9).numpy()
            if beta == 0.0:
                C[:, :, :m] = np.nan  # beta == 0: C must not be read
            ref = oracle.dgemm(ta, tb, m, n, k, alpha, A, B, beta, C)
            Cg = gpu(C)
            with forced(bf, bf.ROUTINE_DGEMM, code2(ta, tb), variant):
                bf.dgemm(ta, tb, alpha, gpu(A), gpu(B), beta, Cg, m=m, n=n, k=k)
            out = host(Cg)
            assert np.isfinite(out[:, :, :m]).all()
            assert normwise(out, ref, m) <= TOL, (m, n, k, ta, tb)


@pytest.mark.parametrize("variant", [0, 1], ids=["direct", "packed"])
def test_dgemm_integer_bit_exact(bf, oracle, variant):
    for n in (4, 12, 24, 48, 96):
        for ta, tb in TRANS:
            A = bfsynth.randint_batch(6, n, n, n + 3, 11).numpy()
            B = bfsynth.randint_batch(6, n, n, n + 3, 12).numpy()
            C = bfsynth.randint_batch(6, n, n, n + 3, 13).numpy()
            ref = oracle.dgemm(ta, tb, n, n, n, 1.0, A, B, 1.0, C)
            Cg = gpu(C)
            with forced(bf, bf.ROUTINE_DGEMM, code2(ta, tb), variant):
                bf.dgemm(ta, tb, 1.0, gpu(A), gpu(B), 1.0, Cg, m=n, n=n, k=n)
            np.testing.assert_array_equal(host(Cg)[:, :, :n], ref[:, :, :n])


def test_dgemm_pointer_array_and_single(bf, oracle):
    import ctypes
    n, batch = 24, 11
    A = bfsynth.randn_batch(batch, n, n, n, 21).numpy()
    B = bfsynth.randn_batch(batch, n, n, n, 22).numpy()
    C = bfsynth.randn_batch(batch, n, n, n, 23).numpy()
    ref = oracle.dgemm("T", "N", n, n, n, 1.0, A, B, 1.0, C)
    Ag, Bg, Cg = gpu(A), gpu(B), gpu(C)
    # reverse the problem order through the pointer arrays
    order = list(range(batch))[::-1]
    pa = torch.tensor([Ag[i].data_ptr() for i in order], dtype=torch.int64, device="cuda")
    pb = torch.tensor([Bg[i].data_ptr() for i in order], dtype=torch.int64, device="cuda")
    pc = torch.tensor([Cg[i].data_ptr() for i in order], dtype=torch.int64, device="cuda")
    st = bf._stream()
    r = bf.bf_dgemm_batched(b"T", b"N", n, n, n, 1.0, ctypes.c_void_p(pa.data_ptr()), n,
                            ctypes.c_void_p(pb.data_ptr()), n, 1.0, ctypes.c_void_p(pc.data_ptr()), n,
                            batch, st)
    assert r == 0
    assert normwise(host(Cg), ref, n) <= TOL
    # the single-matrix entry point
    C1 = gpu(C[:1].copy())
    r = bf.bf_dgemm(b"T", b"N", n, n, n, 1.0, ctypes.c_void_p(Ag.data_ptr()), n,
                    ctypes.c_void_p(Bg.data_ptr()), n, 1.0, ctypes.c_void_p(C1.data_ptr()), n, st)
    assert r == 0
    assert normwise(host(C1), ref[:1], n) <= TOL


def test_dgemm_config_smallest_full(bf, oracle):
    """4096 problems of n = 24, lda = 24: C += A B^T, every problem compared."""
    n, batch, s = 24, 4096, bfsynth.BASE_SEED
    A = bfsynth.randn_batch(batch, n, n, n, s).numpy()
    B = bfsynth.randn_batch(batch, n, n, n, s + 1).numpy()
    C = bfsynth.randn_batch(batch, n, n, n, s + 2).numpy()
    ref = oracle.dgemm("N", "T", n, n, n, 1.0, A, B, 1.0, C)
    Cg = gpu(C)
    bf.dgemm("N", "T", 1.0, gpu(A), gpu(B), 1.0, Cg)
    assert normwise(host(Cg), ref, n) <= TOL


# ----------------------------------------------------------------------------- dtrsm
TRSM_CASES = list(itertools.product("LR", "LU", "NT", "NU"))


def tri_batch(batch, order, ld, uplo, diag, seed):
    """Well-conditioned triangular matrices; the unused triangle (and a unit diagonal) is NaN."""
    g = torch.Generator().manual_seed(seed)
    T = torch.randn((batch, order, order), generator=g, dtype=torch.float64) / np.sqrt(order)
    d = 1.0 + torch.rand((batch, order), generator=g, dtype=torch.float64)
    T = T.numpy()
    out = np.full((batch, order, ld), np.nan)
    for j in range(order):
        for i in range(order):
            keep = (i > j) if uplo == "L" else (i < j)
            if keep:
                out[:, j, i] = T[:, j, i]
            elif i == j and diag == "N":
                out[:, j, i] = d[:, i].numpy() * np.sign(T[:, j, i] + 0.5)
    return out


@pytest.mark.parametrize("variant", [0, 1, 2], ids=["direct", "packed", "blocked"])
@pytest.mark.parametrize("side,uplo,ta,diag", TRSM_CASES)
def test_dtrsm_all_cases(bf, oracle, variant, side, uplo, ta, diag):
    code = (8 if side == "R" else 0) + (4 if uplo == "U" else 0) + (2 if ta == "T" else 0) + (
        1 if diag == "U" else 0)
    for (m, n) in [(24, 24), (5, 13), (13, 5), (67, 33), (1, 4), (100, 70)]:
        for pad in (0, 3):
            order = m if side == "L" else n
            batch = 7
            A = tri_batch(batch, order, order + pad, uplo, diag, 100 + m + n)
            B = bfsynth.randn_batch(batch, m, n, m + pad, 200 + m).numpy()
            alpha = 1.0 if pad == 0 else -0.75
            ref = oracle.dtrsm(side, uplo, ta, diag, m, n, alpha, A, B)
            Bg = gpu(B)
            with forced(bf, bf.ROUTINE_DTRSM, code, variant):
                bf.dtrsm(side, uplo, ta, diag, alpha, gpu(A), Bg, m=m, n=n)
            out = host(Bg)
            assert normwise(out, ref, m) <= TOL, (m, n, pad)
            assert np.isnan(out[:, :, m:]).all()


def test_dtrsm_alpha_zero(bf):
    B = gpu(np.full((3, 4, 5), np.nan))
    A = gpu(np.full((3, 4, 4), np.nan))
    bf.dtrsm("R", "L", "T", "N", 0.0, A, B, m=5, n=4)
    assert (host(B) == 0.0).all()
    # the blocked form (small batch, order >= 64) takes the same path: B = 0, A not read
    B = gpu(np.full((2, 70, 80), np.nan))
    A = gpu(np.full((2, 70, 70), np.nan))
    bf.dtrsm("R", "U", "N", "N", 0.0, A, B, m=80, n=70)
    assert (host(B) == 0.0).all()


# ----------------------------------------------------------------------------- dpotrf
def spd_upper_nan(batch, n, ld, seed):
    S = bfsynth.spd_batch(batch, n, ld, seed).numpy()
    for j in range(n):
        S[:, j, :j] = np.nan  # strict upper triangle: never read, never written
    return S


# (name, variant, T, NB, lane row-block height or team size, lane k-loop unroll); forced for both
# leading-dimension parities (table code -1)
POTRF_VARIANTS = [("direct4u2", 0, 0, 0, 4, 2), ("direct4u1", 0, 64, 0, 4, 1), ("direct8u1", 0, 0, 0, 8, 1),
                  ("direct8u2", 0, 256, 0, 8, 2), ("packed", 1, 128, 0, 0, 0), ("blocked8", 2, 0, 8, 0, 0),
                  ("blocked32", 2, 0, 32, 0, 0), ("cta", 4, 0, 0, 0, 0), ("team2", 5, 0, 0, 2, 0),
                  ("team4", 5, 128, 0, 4, 0), ("group", 6, 0, 0, 0, 0)]


@pytest.mark.parametrize("vname,variant,T,NB,R,U", POTRF_VARIANTS, ids=[v[0] for v in POTRF_VARIANTS])
@pytest.mark.parametrize("n", SMALL_N)
def test_dpotrf(bf, oracle, vname, variant, T, NB, R, U, n):
    if variant == 1 and n > 16:
        pytest.skip("packed lane Cholesky holds whole problems in shared memory (small n)")
    for pad in (0, 3):
        batch = small_batch(n) + 2
        S = spd_upper_nan(batch, n, n + pad, 300 + n + pad)
        L, info = oracle.dpotrf_l(S)
        assert (info == 0).all()
        Sg = gpu(S)
        with forced(bf, bf.ROUTINE_DPOTRF, -1, variant, T, NB, R, U):
            ig = bf.dpotrf(Sg, n=n)
        out = host(Sg)
        assert (host(ig) == 0).all()
        assert normwise(lower_part(out, n), lower_part(L, n), n) <= TOL
        for j in range(n):
            assert np.isnan(out[:, j, :j]).all()
        assert np.isnan(out[:, :, n:]).all()


@pytest.mark.parametrize("vname,variant,T,NB,R,U", POTRF_VARIANTS, ids=[v[0] for v in POTRF_VARIANTS])
def test_dpotrf_failures(bf, oracle, vname, variant, T, NB, R, U):
    for n in (5, 12, 40, 41, 100):
        if variant == 1 and n > 16:
            continue
        batch = 9
        S = spd_upper_nan(batch, n, n, 400 + n)
        # problem 2: negative pivot at column 3; problem 5: NaN at column n; problem 7: zero pivot 1
        S[2, 2, 2] = -50.0 * n
        S[5, n - 1, n - 1] = np.nan
        S[7, 0, 0] = 0.0
        L, info = oracle.dpotrf_l(S)
        Sg = gpu(S)
        with forced(bf, bf.ROUTINE_DPOTRF, -1, variant, T, NB, R, U):
            ig = bf.dpotrf(Sg, n=n)
        gi = host(ig)
        np.testing.assert_array_equal(gi, info)
        ok = info == 0
        assert normwise(lower_part(host(Sg)[ok], n), lower_part(L[ok], n), n) <= TOL


def test_dpotrf_size_switch_batches(bf, oracle):
    """The built-in batch-size switch (no forced entry): one problem per CTA, teams of 4 and of
    2 lanes per problem, the lane form, and the blocked form whose diagonal blocks take the
    team form, each on a sample of the batch compared with the oracle."""
    cases = [(32, 1024), (32, 4096), (24, 9000), (48, 12000), (48, 30000), (32, 40000), (100, 8000)]
    for n, batch in cases:
        for pad in (0, 3):
            Sg = bfsynth.spd_batch(batch, n, n + pad, 700 + n + pad, device="cuda")
            idx = np.unique(np.r_[0, batch - 1, np.random.default_rng(n).integers(0, batch, 6)])
            sel = torch.as_tensor(idx, device="cuda")
            S = host(Sg[sel])
            ig = bf.dpotrf(Sg, n=n)
            assert int(host(ig).max()) == 0 and int(host(ig).min()) == 0
            L, _ = oracle.dpotrf_l(S)
            out = host(Sg[sel])
            assert normwise(lower_part(out, n), lower_part(L, n), n) <= TOL, (n, batch, pad)


@pytest.mark.parametrize("n,batch", [(24, 4096), (24, 4097), (13, 1), (32, 7001), (5, 20000), (64, 20000)])
def test_dpotrf_group_batches(bf, oracle, n, batch):
    """The group form (problems per CTA in shared memory) on the batch sizes it is made for, with
    groups of up to the shared-memory bound, a ragged last group and, at n = 64 x 20000, more
    groups than CTAs (the CTAs loop over groups); failures planted in the middle of groups.
    Sampled problems (and every failing one) against the oracle; every info checked."""
    for pad in (0, 3):
        Sg = bfsynth.spd_batch(batch, n, n + pad, 800 + n + pad, device="cuda")
        bad = sorted({min(batch - 1, 3), batch // 2, batch - 1}) if batch > 1 else []
        for i, q in enumerate(bad):
            j = (i * 7) % n
            Sg[q, j, j] = -1.0 if i % 2 else float("nan")
        idx = np.unique(np.r_[0, batch - 1, bad, np.random.default_rng(n).integers(0, batch, 8)]).astype(np.int64)
        sel = torch.as_tensor(idx, device="cuda")
        S = host(Sg[sel])
        with forced(bf, bf.ROUTINE_DPOTRF, -1, bf.VARIANT_GROUP):
            ig = bf.dpotrf(Sg, n=n)
        L, info = oracle.dpotrf_l(S)
        gi = host(ig)
        np.testing.assert_array_equal(gi[idx], info)
        assert (np.delete(gi, bad) == 0).all()
        ok = info == 0
        out = host(Sg[sel])
        assert normwise(lower_part(out[ok], n), lower_part(L[ok], n), n) <= TOL, (n, batch, pad)
        assert np.array_equal(out[:, :, n:], S[:, :, n:], equal_nan=True)  # padding untouched


def test_dpotrs(bf, oracle):
    for n in (3, 24, 67, 130):
        batch, nrhs = 6, 4
        S = bfsynth.spd_batch(batch, n, n + 1, 500 + n).numpy()
        L, _ = oracle.dpotrf_l(S)
        Bm = bfsynth.randn_batch(batch, n, nrhs, n + 2, 600 + n).numpy()
        ref = oracle.dpotrs_l(L, Bm, n, nrhs)
        Bg = gpu(Bm)
        bf.dpotrs(gpu(L), Bg, n=n, nrhs=nrhs)
        assert normwise(host(Bg), ref, n) <= TOL


# ----------------------------------------------------------------------------- full-size sweep points
def sample_idx(batch, k=12, seed=0):
    rng = np.random.default_rng(seed)
    idx = set([0, batch - 1]) | set(rng.integers(0, batch, k).tolist())
    return np.array(sorted(idx))


@pytest.mark.parametrize("n", bfsynth.SWEEP_N)
@pytest.mark.parametrize("pad", [0, 3])
def test_sweep_full_size_sampled(bf, oracle, n, pad):
    """Full sweep batches (about 2 GiB of operands) in the configuration the benchmark times;
    sampled problems compared with the oracle."""
    ld = n + pad
    # dgemm, all four forms
    batch = bfsynth.sweep_batch(n, ld, 3)
    idx = sample_idx(batch, seed=n)
    A = bfsynth.randn_batch(batch, n, n, ld, 1, device="cuda")
    B = bfsynth.randn_batch(batch, n, n, ld, 2, device="cuda")
    C0 = bfsynth.randn_batch(batch, n, n, ld, 3, device="cuda")
    Ah, Bh, Ch = (host(x[idx]) for x in (A, B, C0))
    for ta, tb in TRANS:
        C = C0.clone()
        bf.dgemm(ta, tb, 1.0, A, B, 1.0, C, m=n, n=n, k=n)
        ref = oracle.dgemm(ta, tb, n, n, n, 1.0, Ah, Bh, 1.0, Ch)
        assert normwise(host(C[idx]), ref, n) <= TOL, (ta, tb)
    del A, B, C0, C
    torch.cuda.empty_cache()
    # dtrsm right-lower-transposed, unit-scaled L (rltu) and L itself (rltn)
    batch = bfsynth.sweep_batch(n, ld, 2)
    idx = sample_idx(batch, seed=n + 1)
    for unit in (True, False):
        L = bfsynth.unit_lower_batch(batch, n, ld, 4, device="cuda", unit=unit)
        X = bfsynth.randn_batch(batch, n, n, ld, 5, device="cuda")
        Lh, Xh = host(L[idx]), host(X[idx])
        d = "U" if unit else "N"
        bf.dtrsm("R", "L", "T", d, 1.0, L, X, m=n, n=n)
        ref = oracle.dtrsm("R", "L", "T", d, n, n, 1.0, Lh, Xh)
        assert normwise(host(X[idx]), ref, n) <= TOL
        del L, X
    torch.cuda.empty_cache()
    # dpotrf on S = G G^T + n I
    batch = bfsynth.sweep_batch(n, ld, 1)
    idx = sample_idx(batch, seed=n + 2)
    S = bfsynth.spd_batch(batch, n, ld, 6, device="cuda")
    Sh = host(S[idx])
    info = bf.dpotrf(S)
    assert int(host(info).max()) == 0 and int(host(info).min()) == 0
    Lr, _ = oracle.dpotrf_l(Sh)
    assert normwise(lower_part(host(S[idx]), n), lower_part(Lr, n), n) <= TOL
    del S
    torch.cuda.empty_cache()
