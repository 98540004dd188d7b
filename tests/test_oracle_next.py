"""Pins for the oracle's dsyrk, fused dsyrk + dpotrf, dtrmm, upper dpotrf, dgetrf / dgetrs
and the square-root Riccati recursion.

Each function is checked against something other than its own arithmetic:
  dsyrk (section 3.1 "dsyrk")   exact integer products (int64 matmul), numpy matmul,
                                BLAS corner cases (beta = 0 with NaN in C, alpha = 0 with
                                NaN in A, k = 0), the other triangle untouched;
  dsyrk + dpotrf (section 5)    numpy's Cholesky of C + A A^T, closed forms, info;
  dtrmm (section 3.1 "dtrmm")   exact integer products for all 16 cases, unit diagonal and
                                the other triangle never read, alpha = 0;
  dpotrf 'U' (appendix table)   numpy's Cholesky transposed, the [-1, 2, -1] closed form,
                                info, lower triangle untouched;
  dgetrf / dgetrs (section 3.1) scipy's LAPACK lu_factor (pivots exact, factors to
                                rounding), P A = L U, a permutation matrix, zero columns,
                                numpy's solve for both transposes;
  Riccati (section 5)           the classical (non-square-root) recursion
                                P = Q + A^T P A - (S^T + A^T P B)(R + B^T P B)^{-1}(S + B^T P A)
                                evaluated with numpy, and its blocks Lambda, L.
"""
import itertools

import numpy as np
import pytest

rng = np.random.default_rng(20190221)


def cm(M, ld=None, fill=np.nan):
    """One matrix (rows x cols) -> oracle batch layout (1, cols, ld)."""
    r, c = M.shape
    ld = r if ld is None else ld
    out = np.full((1, c, ld), fill)
    out[0, :, :r] = M.T
    return out


def dense(X, rows):
    return X[0, :, :rows].T.copy()


# ----------------------------------------------------------------------------- dsyrk
@pytest.mark.parametrize("uplo,trans", list(itertools.product("LU", "NT")))
def test_dsyrk_integer_exact(oracle, uplo, trans):
    n, k = 13, 7
    A = rng.integers(-3, 4, size=(n, k) if trans == "N" else (k, n)).astype(np.float64)
    C = rng.integers(-5, 6, size=(n, n)).astype(np.float64)
    C = C + C.T
    Ai = A.astype(np.int64)
    prod = Ai @ Ai.T if trans == "N" else Ai.T @ Ai
    Cin = C.copy()
    mask = np.tril(np.ones((n, n), bool)) if uplo == "L" else np.triu(np.ones((n, n), bool))
    Cin[~mask] = np.nan  # the other triangle is neither read nor written
    out = dense(oracle.dsyrk(uplo, trans, n, k, 1.0, cm(A, A.shape[0] + 2), 1.0, cm(Cin, n + 1)), n)
    np.testing.assert_array_equal(out[mask], (prod + C.astype(np.int64))[mask].astype(np.float64))
    assert np.isnan(out[~mask]).all()


def test_dsyrk_float_vs_numpy(oracle):
    n, k = 20, 11
    A = rng.standard_normal((n, k))
    C = rng.standard_normal((n, n))
    out = dense(oracle.dsyrk("L", "N", n, k, -0.75, cm(A), 1.5, cm(C)), n)
    ref = -0.75 * (A @ A.T) + 1.5 * C
    low = np.tril(np.ones((n, n), bool))
    assert np.abs(out[low] - ref[low]).max() <= 1e-13 * np.abs(ref).max()
    np.testing.assert_array_equal(out[~low], C[~low])


def test_dsyrk_blas_corners(oracle):
    n, k = 6, 4
    A = rng.standard_normal((n, k))
    Cnan = np.full((n, n), np.nan)
    out = dense(oracle.dsyrk("U", "N", n, k, 2.0, cm(A), 0.0, cm(Cnan)), n)  # beta = 0: C not read
    up = np.triu(np.ones((n, n), bool))
    ref = (2.0 * A @ A.T)[up]
    assert np.abs(out[up] - ref).max() <= 1e-14 * np.abs(ref).max()
    Anan = np.full((n, k), np.nan)
    C = rng.standard_normal((n, n))
    out = dense(oracle.dsyrk("L", "N", n, k, 0.0, cm(Anan), 3.0, cm(C)), n)  # alpha = 0: A not read
    low = np.tril(np.ones((n, n), bool))
    np.testing.assert_array_equal(out[low], 3.0 * C[low])
    out = dense(oracle.dsyrk("L", "T", n, 0, 1.0, cm(np.zeros((1, n))), 0.5, cm(C)), n)  # k = 0
    np.testing.assert_array_equal(out[low], 0.5 * C[low])


# ----------------------------------------------------------------------------- dsyrk + dpotrf
def test_dsyrk_dpotrf_vs_numpy_cholesky(oracle):
    n, k = 17, 9
    A = rng.standard_normal((n, k))
    G = rng.standard_normal((n, n))
    C = G @ G.T + n * np.eye(n)
    Cin = C.copy()
    Cin[np.triu_indices(n, 1)] = np.nan
    F, info = oracle.dsyrk_dpotrf_l(n, k, cm(A), cm(Cin, n + 2))
    assert info[0] == 0
    L = np.tril(dense(F, n))
    Lref = np.linalg.cholesky(C + A @ A.T)
    assert np.abs(L - Lref).max() <= 1e-13 * np.abs(Lref).max()
    assert np.isnan(dense(F, n)[np.triu_indices(n, 1)]).all()


def test_dsyrk_dpotrf_closed_forms_and_info(oracle):
    n = 5
    F, info = oracle.dsyrk_dpotrf_l(n, 1, cm(np.zeros((n, 1))), cm(np.eye(n)))
    np.testing.assert_array_equal(np.tril(dense(F, n)), np.eye(n))
    e0 = np.zeros((n, 1))
    e0[0, 0] = 1.0
    F, info = oracle.dsyrk_dpotrf_l(n, 1, cm(e0), cm(np.eye(n)))  # chol(I + e0 e0^T) = diag(sqrt 2, 1, ...)
    ref = np.eye(n)
    ref[0, 0] = np.sqrt(2.0)
    np.testing.assert_array_equal(np.tril(dense(F, n)), ref)
    C = np.eye(n)
    C[2, 2] = -1.0
    _, info = oracle.dsyrk_dpotrf_l(n, 1, cm(np.zeros((n, 1))), cm(C))
    assert info[0] == 3


# ----------------------------------------------------------------------------- dtrmm
def tri_dense(A, uplo, trans, diag):
    T = np.tril(A) if uplo == "L" else np.triu(A)
    if diag == "U":
        np.fill_diagonal(T, 1)
    return T.T if trans == "T" else T


@pytest.mark.parametrize("side,uplo,trans,diag", list(itertools.product("LR", "LU", "NT", "NU")))
def test_dtrmm_integer_exact(oracle, side, uplo, trans, diag):
    m, n = 9, 7
    k = m if side == "L" else n
    A = rng.integers(-3, 4, size=(k, k)).astype(np.float64)
    B = rng.integers(-4, 5, size=(m, n)).astype(np.float64)
    Astore = A.copy()
    other = np.triu_indices(k, 1) if uplo == "L" else np.tril_indices(k, -1)
    Astore[other] = np.nan  # the other triangle is never read
    if diag == "U":
        np.fill_diagonal(Astore, np.nan)  # nor the unit diagonal
    T = tri_dense(A.astype(np.int64), uplo, trans, diag)
    Bi = B.astype(np.int64)
    ref = 2 * (T @ Bi if side == "L" else Bi @ T)
    out = dense(oracle.dtrmm(side, uplo, trans, diag, m, n, 2.0, cm(Astore, k + 1), cm(B, m + 3)), m)
    np.testing.assert_array_equal(out, ref.astype(np.float64))


def test_dtrmm_alpha_zero(oracle):
    m, n = 4, 6
    out = oracle.dtrmm("R", "L", "N", "N", m, n, 0.0, cm(np.full((n, n), np.nan)), cm(np.full((m, n), np.nan)))
    np.testing.assert_array_equal(dense(out, m), np.zeros((m, n)))


# ----------------------------------------------------------------------------- dpotrf upper
def test_dpotrf_u_vs_numpy(oracle):
    n = 23
    G = rng.standard_normal((n, n))
    S = G @ G.T + n * np.eye(n)
    Sin = S.copy()
    Sin[np.tril_indices(n, -1)] = np.nan  # only the upper triangle is read
    U, info = oracle.dpotrf_u(cm(Sin, n + 1))
    assert info[0] == 0
    Ur = np.linalg.cholesky(S).T
    out = dense(U, n)
    assert np.abs(np.triu(out) - Ur).max() <= 1e-13 * np.abs(Ur).max()
    assert np.isnan(out[np.tril_indices(n, -1)]).all()


def test_dpotrf_u_tridiagonal_closed_form(oracle):
    n = 12
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    U, info = oracle.dpotrf_u(cm(T))
    i = np.arange(1, n + 1)
    ref = np.diag(np.sqrt((i + 1) / i)) + np.diag(-np.sqrt(i[:-1] / (i[:-1] + 1)), k=1)
    np.testing.assert_allclose(np.triu(dense(U, n)), ref, rtol=1e-14, atol=1e-15)


def test_dpotrf_u_info(oracle):
    A = np.eye(6)
    A[3, 3] = -2.0
    _, info = oracle.dpotrf_u(cm(A))
    assert info[0] == 4


# ----------------------------------------------------------------------------- dgetrf / dgetrs
def test_dgetrf_vs_lapack(oracle):
    sl = pytest.importorskip("scipy.linalg")
    for n in (1, 2, 5, 16, 33):
        A = rng.standard_normal((n, n))
        LU, ipiv, info = oracle.dgetrf(cm(A, n + 2), m=n)
        assert info[0] == 0
        lu_ref, piv_ref = sl.lu_factor(A)
        np.testing.assert_array_equal(ipiv[0], piv_ref + 1)
        got = dense(LU, n)
        assert np.abs(got - lu_ref).max() <= 1e-12 * max(1.0, np.abs(lu_ref).max())


def test_dgetrf_reconstruction(oracle):
    n = 20
    A = rng.standard_normal((n, n))
    LU, ipiv, info = oracle.dgetrf(cm(A), m=n)
    F = dense(LU, n)
    L = np.tril(F, -1) + np.eye(n)
    U = np.triu(F)
    PA = A.copy()
    for j, p in enumerate(ipiv[0] - 1):  # apply the row swaps in order
        PA[[j, p]] = PA[[p, j]]
    assert np.abs(PA - L @ U).max() <= 1e-13 * np.abs(A).max() * n
    assert (np.abs(np.tril(F, -1)) <= 1.0).all()  # partial pivoting: |l_ij| <= 1


def test_dgetrf_permutation_and_zero_column(oracle):
    n = 6
    perm = np.array([3, 0, 5, 1, 4, 2])
    P = np.eye(n)[perm]  # row i of P is e_{perm[i]}
    LU, ipiv, info = oracle.dgetrf(cm(P), m=n)
    F = dense(LU, n)
    assert info[0] == 0
    np.testing.assert_array_equal(np.tril(F, -1), np.zeros((n, n)))
    np.testing.assert_array_equal(np.abs(np.diag(F)), np.ones(n))
    A = rng.standard_normal((n, n))
    A[:, 2] = 0.0  # after elimination the pivot column 2 is exactly zero
    A[:, 3] = A[:, 1]
    _, _, info = oracle.dgetrf(cm(A), m=n)
    assert info[0] == 3


@pytest.mark.parametrize("trans", "NT")
def test_dgetrs_vs_numpy(oracle, trans):
    n, r = 19, 3
    A = rng.standard_normal((n, n)) + 3 * np.eye(n)
    B = rng.standard_normal((n, r))
    LU, ipiv, info = oracle.dgetrf(cm(A), m=n)
    X = dense(oracle.dgetrs(trans, LU, ipiv, cm(B), n, r), n)
    ref = np.linalg.solve(A if trans == "N" else A.T, B)
    assert np.abs(X - ref).max() <= 1e-12 * np.abs(ref).max()


# ----------------------------------------------------------------------------- Riccati
def riccati_inputs(N, nx, nu, seed):
    g = np.random.default_rng(seed)
    m = nx + nu
    A = g.standard_normal((N, nx, nx)) / np.sqrt(nx)
    B = g.standard_normal((N, nx, nu)) / np.sqrt(nx)
    G = g.standard_normal((N, m, m))
    RSQ = G @ np.transpose(G, (0, 2, 1)) + m * np.eye(m)
    H = g.standard_normal((nx, nx))
    QN = H @ H.T + nx * np.eye(nx)
    BAt = np.concatenate([np.transpose(B, (0, 2, 1)), np.transpose(A, (0, 2, 1))], axis=1)  # (N, m, nx)
    return A, B, RSQ, QN, BAt


@pytest.mark.parametrize("nx,nu", [(8, 4), (24, 12)])
def test_riccati_vs_classical_recursion(oracle, nx, nu):
    N = 10
    m = nx + nu
    A, B, RSQ, QN, BAt = riccati_inputs(N, nx, nu, 7 + nx)
    F, info = oracle.riccati(np.transpose(BAt, (0, 2, 1))[None].copy(),
                             np.transpose(RSQ, (0, 2, 1))[None].copy(), QN.T[None].copy(), nx, nu)
    assert info[0] == 0
    P = QN.copy()
    Lc = np.tril(F[0, N].T[:nx, :nx])
    np.testing.assert_allclose(Lc @ Lc.T, P, rtol=1e-12, atol=1e-12 * np.abs(P).max())
    for s in range(N - 1, -1, -1):
        R, S, Q = RSQ[s][:nu, :nu], RSQ[s][:nu, nu:], RSQ[s][nu:, nu:]
        As, Bs = A[s], B[s]
        Rt = R + Bs.T @ P @ Bs
        St = S + Bs.T @ P @ As
        P = Q + As.T @ P @ As - St.T @ np.linalg.solve(Rt, St)
        P = 0.5 * (P + P.T)
        Fs = np.tril(F[0, s].T)
        Lam, Ls, Lc = Fs[:nu, :nu], Fs[nu:, :nu], Fs[nu:, nu:]
        tol = 1e-11 * np.abs(P).max()
        np.testing.assert_allclose(Lc @ Lc.T, P, rtol=1e-11, atol=tol)  # the Riccati matrix P_s
        np.testing.assert_allclose(Lam @ Lam.T, Rt, rtol=1e-11, atol=1e-11 * np.abs(Rt).max())
        np.testing.assert_allclose(Ls @ Lam.T, St.T, rtol=1e-11, atol=1e-11 * np.abs(St).max())


def test_riccati_zero_dynamics(oracle):
    # A = 0, B = 0: every stage factor is chol([R S; S^T Q])
    N, nx, nu = 3, 4, 2
    m = nx + nu
    _, _, RSQ, QN, _ = riccati_inputs(N, nx, nu, 3)
    BAt = np.zeros((1, N, nx, m))
    F, info = oracle.riccati(BAt, np.transpose(RSQ, (0, 2, 1))[None].copy(), QN.T[None].copy(), nx, nu)
    for s in range(N):
        np.testing.assert_allclose(np.tril(F[0, s].T), np.linalg.cholesky(RSQ[s]), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("m,n", [(7, 3), (3, 7), (33, 17), (17, 33), (1, 5), (5, 1), (40, 40)])
def test_dgetrf_rectangular(oracle, m, n):
    """m x n LU (section 3.1 "dgetrf" is an m x n routine): pivots identical to LAPACK's (scipy's
    lu_factor), factors within rounding, and P A = L U with L m x min(m, n) unit lower
    trapezoidal, U min(m, n) x n upper trapezoidal, |l_ij| <= 1; padding rows untouched."""
    sl = pytest.importorskip("scipy.linalg")
    A = rng.standard_normal((m, n))
    k = min(m, n)
    LU, ipiv, info = oracle.dgetrf(cm(A, m + 3), m=m, n=n)
    assert info[0] == 0 and ipiv.shape == (1, k)
    assert np.isnan(LU[0, :, m:]).all()
    lu_ref, piv_ref = sl.lu_factor(A)
    np.testing.assert_array_equal(ipiv[0], piv_ref + 1)
    F = dense(LU, m)
    assert np.abs(F - lu_ref).max() <= 1e-12 * max(1.0, np.abs(lu_ref).max())
    L = np.tril(F[:, :k], -1) + np.eye(m, k)
    U = np.triu(F[:k, :])
    PA = A.copy()
    for j, p in enumerate(ipiv[0] - 1):
        PA[[j, p]] = PA[[p, j]]
    assert np.abs(PA - L @ U).max() <= 1e-13 * np.abs(A).max() * max(m, n)
    assert (np.abs(L) <= 1.0).all()
