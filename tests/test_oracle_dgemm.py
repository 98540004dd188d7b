"""Pins for the oracle's dgemm (section 2.1: C <= alpha op(A) op(B) + beta C).

Nothing here re-types the oracle's loop: the checks are hand-expanded 2x2 and
3x3 formulas, exact integer products computed with Python integers,
special cases (identity, diagonal, alpha = 0, beta = 0 with NaN in C) and the
transposition identity (A B)^T = B^T A^T that the paper uses for the 'TT'
direct kernel (section 2.2, algorithm 'D').
"""
import itertools

import numpy as np
import pytest

TRANS = ["N", "T"]


def colmajor(M, ld=None):
    """(rows, cols) row-major numpy -> (1, cols, ld) column-major batch."""
    r, c = M.shape
    ld = r if ld is None else ld
    out = np.full((1, c, ld), np.nan)
    out[0, :, :r] = M.T
    return out


def from_colmajor(X, rows):
    return X[0, :, :rows].T.copy()


def op(M, t):
    return M if t == "N" else M.T


@pytest.mark.parametrize("ta,tb", list(itertools.product(TRANS, TRANS)))
def test_2x2_expansion(oracle, ta, tb):
    a11, a21, a12, a22 = 1.5, -2.0, 0.25, 3.0
    b11, b21, b12, b22 = -1.0, 0.5, 2.0, -0.75
    c11, c21, c12, c22 = 0.125, 1.0, -3.0, 2.5
    alpha, beta = 2.0, -0.5
    A = np.array([[a11, a12], [a21, a22]])
    B = np.array([[b11, b12], [b21, b22]])
    C = np.array([[c11, c12], [c21, c22]])
    # op(A), op(B) entries written out by hand
    oa = {("N", 1, 1): a11, ("N", 1, 2): a12, ("N", 2, 1): a21, ("N", 2, 2): a22,
          ("T", 1, 1): a11, ("T", 1, 2): a21, ("T", 2, 1): a12, ("T", 2, 2): a22}
    ob = {("N", 1, 1): b11, ("N", 1, 2): b12, ("N", 2, 1): b21, ("N", 2, 2): b22,
          ("T", 1, 1): b11, ("T", 1, 2): b21, ("T", 2, 1): b12, ("T", 2, 2): b22}
    expect = np.empty((2, 2))
    for i in (1, 2):
        for j in (1, 2):
            s = oa[(ta, i, 1)] * ob[(tb, 1, j)] + oa[(ta, i, 2)] * ob[(tb, 2, j)]
            expect[i - 1, j - 1] = alpha * s + beta * C[i - 1, j - 1]
    got = oracle.dgemm(ta, tb, 2, 2, 2, alpha, colmajor(A), colmajor(B), beta, colmajor(C))
    np.testing.assert_array_equal(from_colmajor(got, 2), expect)


def test_3x3_expansion_nn(oracle):
    # entries chosen so every product and sum is exact in binary64
    A = np.array([[1., 2., 3.], [4., 5., 6.], [7., 8., 10.]])
    B = np.array([[2., 0., 1.], [1., 3., -1.], [0., -2., 4.]])
    # hand expansion of A @ B
    AB = np.array([
        [1*2 + 2*1 + 3*0, 1*0 + 2*3 + 3*-2, 1*1 + 2*-1 + 3*4],
        [4*2 + 5*1 + 6*0, 4*0 + 5*3 + 6*-2, 4*1 + 5*-1 + 6*4],
        [7*2 + 8*1 + 10*0, 7*0 + 8*3 + 10*-2, 7*1 + 8*-1 + 10*4],
    ], dtype=float)
    C0 = np.ones((3, 3))
    got = oracle.dgemm("N", "N", 3, 3, 3, 1.0, colmajor(A), colmajor(B), 1.0, colmajor(C0))
    np.testing.assert_array_equal(from_colmajor(got, 3), AB + 1.0)


@pytest.mark.parametrize("ta,tb", list(itertools.product(TRANS, TRANS)))
@pytest.mark.parametrize("m,n,k,pad", [(24, 24, 24, 0), (7, 5, 11, 3), (1, 9, 4, 1), (13, 13, 1, 2)])
def test_integer_exact(oracle, ta, tb, m, n, k, pad):
    """Integer entries in [-3, 3]: the result is exact, compared with Python integers."""
    rng = np.random.default_rng(1000 + m * 31 + n * 7 + k)
    Ar, Ac = (m, k) if ta == "N" else (k, m)
    Br, Bc = (k, n) if tb == "N" else (n, k)
    A = rng.integers(-3, 4, (Ar, Ac))
    B = rng.integers(-3, 4, (Br, Bc))
    C = rng.integers(-3, 4, (m, n))
    alpha, beta = 3, -2
    oA, oB = op(A, ta).tolist(), op(B, tb).tolist()
    expect = [[alpha * sum(int(oA[i][p]) * int(oB[p][j]) for p in range(k)) + beta * int(C[i][j])
               for j in range(n)] for i in range(m)]
    got = oracle.dgemm(ta, tb, m, n, k, float(alpha), colmajor(A.astype(float), Ar + pad),
                       colmajor(B.astype(float), Br + pad), float(beta),
                       colmajor(C.astype(float), m + pad))
    np.testing.assert_array_equal(from_colmajor(got, m), np.array(expect, dtype=float))
    # the padding rows of C are untouched (still NaN)
    if pad:
        assert np.isnan(got[0, :, m:]).all()


@pytest.mark.parametrize("tb", TRANS)
def test_identity_left(oracle, tb):
    rng = np.random.default_rng(5)
    n = 9
    B = rng.standard_normal((n, n))
    C = rng.standard_normal((n, n))
    got = oracle.dgemm("N", tb, n, n, n, 0.75, colmajor(np.eye(n)), colmajor(B), 0.5, colmajor(C))
    np.testing.assert_array_equal(from_colmajor(got, n), 0.75 * op(B, tb) + 0.5 * C)


def test_diagonal_factors(oracle):
    d1 = np.arange(1.0, 7.0)
    d2 = np.linspace(-2, 3, 6)
    got = oracle.dgemm("T", "T", 6, 6, 6, 1.0, colmajor(np.diag(d1)), colmajor(np.diag(d2)), 0.0,
                       colmajor(np.full((6, 6), np.nan)))
    np.testing.assert_array_equal(from_colmajor(got, 6), np.diag(d1 * d2))


def test_beta_zero_does_not_read_c(oracle):
    rng = np.random.default_rng(6)
    A, B = rng.standard_normal((4, 4)), rng.standard_normal((4, 4))
    C = np.full((4, 4), np.nan)
    got = oracle.dgemm("N", "N", 4, 4, 4, 1.0, colmajor(A), colmajor(B), 0.0, colmajor(C))
    assert np.isfinite(from_colmajor(got, 4)).all()


def test_alpha_zero_scales_only(oracle):
    rng = np.random.default_rng(7)
    A, B, C = (rng.standard_normal((5, 5)) for _ in range(3))
    got = oracle.dgemm("N", "T", 5, 5, 5, 0.0, colmajor(A), colmajor(B), 2.0, colmajor(C))
    np.testing.assert_array_equal(from_colmajor(got, 5), 2.0 * C)


def test_tt_is_transposed_nn(oracle):
    """(B A)^T computed by 'NN' equals A^T B^T computed by 'TT' bit for bit (section 2.2 'D')."""
    rng = np.random.default_rng(8)
    n = 17
    A, B = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    Z = np.zeros((n, n))
    tt = from_colmajor(oracle.dgemm("T", "T", n, n, n, 1.0, colmajor(A), colmajor(B), 0.0,
                                    colmajor(Z)), n)
    nn = from_colmajor(oracle.dgemm("N", "N", n, n, n, 1.0, colmajor(B), colmajor(A), 0.0,
                                    colmajor(Z)), n)
    np.testing.assert_array_equal(tt, nn.T)


def test_nt_equals_nn_with_explicit_transpose(oracle):
    rng = np.random.default_rng(9)
    n = 12
    A, B = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    Z = np.zeros((n, n))
    nt = oracle.dgemm("N", "T", n, n, n, 1.0, colmajor(A), colmajor(B), 0.0, colmajor(Z))
    nn = oracle.dgemm("N", "N", n, n, n, 1.0, colmajor(A), colmajor(B.T.copy()), 0.0, colmajor(Z))
    np.testing.assert_array_equal(nt, nn)


def test_batched_matches_library_matmul(oracle):
    """Extra cross-check against numpy's matmul on a float batch."""
    rng = np.random.default_rng(10)
    bsz, n = 8, 24
    A = rng.standard_normal((bsz, n, n))
    B = rng.standard_normal((bsz, n, n))
    C = rng.standard_normal((bsz, n, n))
    got = oracle.dgemm("N", "T", n, n, n, 1.0, A, B, 1.0, C)
    # column-major (b, j, i): as row-major matrices these are the transposes
    Am, Bm, Cm = (x.transpose(0, 2, 1) for x in (A, B, C))
    ref = Am @ Bm.transpose(0, 2, 1) + Cm
    np.testing.assert_allclose(got.transpose(0, 2, 1), ref, rtol=0, atol=1e-12)
