"""Pins for the oracle's dpotrf (lower), dtrsm and dpotrs.

Cholesky (section 3.1 "dpotrf"): identity, diagonal, the closed form of the
tridiagonal [-1, 2, -1] factor, the hand-expanded 2x2 and 3x3 formulas,
exact recovery of an integer factor L0 from L0 L0^T, the invariants
L L^T = A / lower / positive diagonal, LAPACK's info on non-SPD input, and
untouched upper triangle and padding.  Triangular solves (section 3.1
"dtrsm", all side/uplo/trans/diag cases): exact recovery of an integer
solution, identity matrix, unit diagonal not read, residual of float cases.
"""
import itertools
import math

import numpy as np
import pytest


def colmajor(M, ld=None, fill=np.nan):
    r, c = M.shape
    ld = r if ld is None else ld
    out = np.full((1, c, ld), fill)
    out[0, :, :r] = M.T
    return out


def from_colmajor(X, rows):
    return X[0, :, :rows].T.copy()


def lower_of(X, n):
    return np.tril(from_colmajor(X, n))


# ----------------------------------------------------------------------------- dpotrf
def test_identity(oracle):
    L, info = oracle.dpotrf_l(colmajor(np.eye(7)))
    assert info[0] == 0
    np.testing.assert_array_equal(lower_of(L, 7), np.eye(7))


def test_diagonal(oracle):
    d = np.array([4.0, 9.0, 2.0, 0.25, 1e-6])
    L, info = oracle.dpotrf_l(colmajor(np.diag(d)))
    assert info[0] == 0
    np.testing.assert_array_equal(np.diag(lower_of(L, 5)), np.sqrt(d))
    np.testing.assert_array_equal(lower_of(L, 5) - np.diag(np.diag(lower_of(L, 5))), 0)


@pytest.mark.parametrize("n", [1, 2, 5, 24, 64])
def test_tridiagonal_closed_form(oracle, n):
    """tridiag(-1, 2, -1): L_ii = sqrt((i+1)/i), L_{i+1,i} = -sqrt(i/(i+1)) (1-based i)."""
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    L, info = oracle.dpotrf_l(colmajor(T))
    assert info[0] == 0
    expect = np.zeros((n, n))
    for i in range(1, n + 1):
        expect[i - 1, i - 1] = math.sqrt((i + 1) / i)
        if i < n:
            expect[i, i - 1] = -math.sqrt(i / (i + 1))
    np.testing.assert_allclose(lower_of(L, n), expect, rtol=4e-16 * n, atol=4e-16 * n)


def test_2x2_closed_form(oracle):
    a, b, c = 4.0, 2.0, 5.0
    L, info = oracle.dpotrf_l(colmajor(np.array([[a, b], [b, c]])))
    l11 = math.sqrt(a)
    l21 = b / l11
    l22 = math.sqrt(c - l21 * l21)
    np.testing.assert_array_equal(lower_of(L, 2), np.array([[l11, 0], [l21, l22]]))


def test_3x3_expansion(oracle):
    A = np.array([[25.0, 15.0, -5.0], [15.0, 18.0, 0.0], [-5.0, 0.0, 11.0]])
    # textbook example: L = [[5,0,0],[3,3,0],[-1,1,3]]
    l11 = math.sqrt(A[0, 0])
    l21 = A[1, 0] / l11
    l31 = A[2, 0] / l11
    l22 = math.sqrt(A[1, 1] - l21 ** 2)
    l32 = (A[2, 1] - l31 * l21) / l22
    l33 = math.sqrt(A[2, 2] - l31 ** 2 - l32 ** 2)
    expect = np.array([[l11, 0, 0], [l21, l22, 0], [l31, l32, l33]])
    np.testing.assert_array_equal(expect, [[5, 0, 0], [3, 3, 0], [-1, 1, 3]])
    L, info = oracle.dpotrf_l(colmajor(A))
    np.testing.assert_array_equal(lower_of(L, 3), expect)


@pytest.mark.parametrize("n,pad", [(6, 0), (24, 3), (40, 1)])
def test_integer_factor_recovered_exactly(oracle, n, pad):
    """A = L0 L0^T with integer L0 (positive integer diagonal): chol(A) = L0 bit for bit."""
    rng = np.random.default_rng(n)
    L0 = np.tril(rng.integers(-3, 4, (n, n)), -1) + np.diag(rng.integers(1, 5, n))
    A = [[sum(int(L0[i, p]) * int(L0[j, p]) for p in range(n)) for j in range(n)] for i in range(n)]
    A = np.array(A, dtype=float)
    Ain = colmajor(A, n + pad)
    # poison the strict upper triangle: only the lower triangle may be read
    for j in range(n):
        Ain[0, j, :j] = np.nan
    L, info = oracle.dpotrf_l(Ain)
    assert info[0] == 0
    np.testing.assert_array_equal(lower_of(np.nan_to_num(L, nan=0.0), n), L0.astype(float))
    # strict upper triangle and padding rows untouched
    for j in range(n):
        assert np.isnan(L[0, j, :j]).all()
    assert np.isnan(L[0, :, n:]).all()


@pytest.mark.parametrize("n", [3, 24, 100])
def test_invariants_random_spd(oracle, n):
    rng = np.random.default_rng(50 + n)
    G = rng.standard_normal((n, n))
    S = G @ G.T + n * np.eye(n)
    L, info = oracle.dpotrf_l(colmajor(S))
    Lm = lower_of(L, n)
    assert info[0] == 0
    assert (np.diag(Lm) > 0).all()
    u = 2.0 ** -53
    assert np.linalg.norm(S - Lm @ Lm.T) / np.linalg.norm(S) <= 4 * n * u
    # cross-check with LAPACK through numpy (extra)
    np.testing.assert_allclose(Lm, np.linalg.cholesky(S), rtol=0, atol=1e-12 * np.abs(Lm).max())


def test_not_positive_definite_info(oracle):
    D = np.diag([1.0, -1.0, 2.0, 3.0])
    _, info = oracle.dpotrf_l(colmajor(D))
    assert info[0] == 2
    M = np.array([[1.0, 2.0], [2.0, 1.0]])  # eigenvalues 3 and -1
    _, info = oracle.dpotrf_l(colmajor(M))
    assert info[0] == 2
    Z = np.zeros((3, 3))
    _, info = oracle.dpotrf_l(colmajor(Z))
    assert info[0] == 1
    N = np.eye(3)
    N[1, 1] = np.nan
    _, info = oracle.dpotrf_l(colmajor(N))
    assert info[0] == 2


def test_batch_mixed_failures(oracle):
    good = np.eye(4) * 4
    bad = np.diag([1.0, 1.0, -1.0, 1.0])
    A = np.concatenate([colmajor(good), colmajor(bad), colmajor(good)], axis=0)
    L, info = oracle.dpotrf_l(A)
    np.testing.assert_array_equal(info, [0, 3, 0])
    np.testing.assert_array_equal(lower_of(L[2:3], 4), 2 * np.eye(4))


def test_n_zero(oracle):
    A = np.zeros((2, 0, 1))
    L, info = oracle.dpotrf_l(A, n=0)
    np.testing.assert_array_equal(info, [0, 0])


# ----------------------------------------------------------------------------- dtrsm
CASES = list(itertools.product("LR", "LU", "NT", "NU"))


def make_tri(rng, n, uplo, diag):
    if uplo == "L":
        T = np.tril(rng.integers(-3, 4, (n, n)), -1)
    else:
        T = np.triu(rng.integers(-3, 4, (n, n)), 1)
    if diag == "U":
        T = T + np.eye(n, dtype=int)
    else:
        T = T + np.diag(rng.choice([-2, -1, 1, 2], n))
    return T


def int_matmul(X, Y):
    X, Y = X.tolist(), Y.tolist()
    return np.array([[sum(int(X[i][p]) * int(Y[p][j]) for p in range(len(Y)))
                      for j in range(len(Y[0]))] for i in range(len(X))], dtype=object)


@pytest.mark.parametrize("side,uplo,ta,diag", CASES)
@pytest.mark.parametrize("m,n", [(5, 5), (7, 3), (2, 9)])
def test_trsm_integer_exact(oracle, side, uplo, ta, diag, m, n):
    """Choose an integer X, form alpha B = op(T) X (left) or X op(T) (right) exactly; solve.

    With a unit diagonal every intermediate is an integer; with a +-1/+-2
    diagonal, X is drawn as a multiple of 2^(order) so every division is exact.
    """
    rng = np.random.default_rng(hash((side, uplo, ta, diag, m, n)) & 0xFFFF)
    order = m if side == "L" else n
    T = make_tri(rng, order, uplo, diag)
    X = rng.integers(-4, 5, (m, n)) * (1 if diag == "U" else 2 ** order)
    opT = T if ta == "N" else T.T
    alpha = 2
    prod = int_matmul(opT, X) if side == "L" else int_matmul(X, opT)
    B = np.array([[int(v) // alpha if int(v) % alpha == 0 else None for v in row] for row in prod],
                 dtype=object)
    if any(v is None for row in B for v in row):
        X = X * alpha
        prod = int_matmul(opT, X) if side == "L" else int_matmul(X, opT)
        B = np.array([[int(v) // alpha for v in row] for row in prod], dtype=object)
    Tin = colmajor(T.astype(float), order + 1)
    # poison the unused triangle, and the diagonal for unit solves
    for j in range(order):
        for i in range(order):
            if (uplo == "L" and i < j) or (uplo == "U" and i > j) or (diag == "U" and i == j):
                Tin[0, j, i] = np.nan
    got = oracle.dtrsm(side, uplo, ta, diag, m, n, float(alpha), Tin,
                       colmajor(B.astype(float), m + 2))
    np.testing.assert_array_equal(from_colmajor(got, m), X.astype(float))
    assert np.isnan(got[0, :, m:]).all()


@pytest.mark.parametrize("side,uplo,ta,diag", CASES)
def test_trsm_identity(oracle, side, uplo, ta, diag):
    rng = np.random.default_rng(3)
    m, n = 6, 4
    B = rng.standard_normal((m, n))
    order = m if side == "L" else n
    got = oracle.dtrsm(side, uplo, ta, diag, m, n, -1.5, colmajor(np.eye(order)), colmajor(B))
    np.testing.assert_array_equal(from_colmajor(got, m), -1.5 * B)


@pytest.mark.parametrize("side,uplo,ta,diag", CASES)
def test_trsm_residual_float(oracle, side, uplo, ta, diag):
    rng = np.random.default_rng(11)
    m, n = 24, 24
    order = m if side == "L" else n
    T = rng.standard_normal((order, order)) / np.sqrt(order)
    T = np.tril(T) if uplo == "L" else np.triu(T)
    np.fill_diagonal(T, 1.0 if diag == "U" else 1.0 + rng.random(order))
    B = rng.standard_normal((m, n))
    X = from_colmajor(oracle.dtrsm(side, uplo, ta, diag, m, n, 1.0, colmajor(T), colmajor(B)), m)
    opT = T if ta == "N" else T.T
    R = (opT @ X if side == "L" else X @ opT) - B
    assert np.linalg.norm(R) / np.linalg.norm(B) < 1e-12


# ----------------------------------------------------------------------------- dpotrs
def test_potrs_integer_exact(oracle):
    rng = np.random.default_rng(21)
    n, r = 8, 4
    L0 = np.tril(rng.integers(-2, 3, (n, n)), -1) + np.eye(n, dtype=int)
    X = rng.integers(-5, 6, (n, r))
    A = int_matmul(L0, L0.T)
    B = int_matmul(A, X)
    got = oracle.dpotrs_l(colmajor(L0.astype(float)), colmajor(B.astype(float)), n, r)
    np.testing.assert_array_equal(from_colmajor(got, n), X.astype(float))


def test_ragged_matches_uniform(oracle):
    rng = np.random.default_rng(31)
    ns = np.array([3, 1, 7, 2, 5], dtype=np.int32)
    nrhs = 4
    offS = np.concatenate([[0], np.cumsum(ns.astype(np.int64) ** 2)[:-1]])
    offX = np.concatenate([[0], np.cumsum(ns.astype(np.int64) * nrhs)[:-1]])
    S = np.zeros(int((ns.astype(np.int64) ** 2).sum()))
    X = rng.standard_normal(int(ns.sum()) * nrhs)
    mats = []
    for b, n in enumerate(ns):
        G = rng.standard_normal((n, n))
        M = G @ G.T + n * np.eye(n)
        mats.append(M)
        S[offS[b]:offS[b] + n * n] = M.T.reshape(-1)
    Sout, Xout, info = oracle.ragged_potrf_potrs(ns, S, offS, X, offX, nrhs)
    assert (info == 0).all()
    for b, n in enumerate(ns):
        L, _ = oracle.dpotrf_l(colmajor(mats[b]))
        np.testing.assert_array_equal(np.tril(Sout[offS[b]:offS[b] + n * n].reshape(n, n).T),
                                      lower_of(L, n))
        Bb = X[offX[b]:offX[b] + n * nrhs].reshape(nrhs, n).T
        ref = from_colmajor(oracle.dpotrs_l(L, colmajor(Bb), n, nrhs), n)
        np.testing.assert_array_equal(Xout[offX[b]:offX[b] + n * nrhs].reshape(nrhs, n).T, ref)
        np.testing.assert_allclose(mats[b] @ ref, Bb, atol=1e-10)
