"""Pins for the oracle's backward error, mixed-precision solve and gradients.

* backward error (Rigal-Gaches): a hand-computed 2x2 case and exact solutions;
* mixed-precision solve: a diagonal system with a closed-form solution,
  backward error <= 1e-12 at cond 1e2..1e6, iteration counts that grow with
  the condition number, binary64 fallback when the binary32 factor fails;
* Cholesky adjoint: central finite differences of a scalar loss, the n = 1
  closed form d sqrt(a)/da = 1/(2 sqrt(a)), and Murray's published matrix
  form evaluated independently with numpy;
* closed-form SPD-solve gradient: central finite differences in J, Q, B.
"""
import math

import numpy as np
import pytest


def colmajor(M, ld=None):
    r, c = M.shape
    ld = r if ld is None else ld
    out = np.full((1, c, ld), np.nan)
    out[0, :, :r] = M.T
    return out


def test_backward_error_hand_case(oracle):
    A = np.array([[2.0, 1.0], [1.0, 3.0]])
    x = np.array([1.0, 1.0])
    b = np.array([3.0, 5.0])
    # r = b - A x = (0, 1); ||r|| = 1, ||A||_inf = 4, ||x|| = 1, ||b|| = 5 -> 1/9
    eta = oracle.backward_error(colmajor(A), x, b)
    assert eta[0] == pytest.approx(1.0 / 9.0, rel=1e-15)
    eta0 = oracle.backward_error(colmajor(A), np.array([0.8, 1.4]), np.array([3.0, 5.0]))
    assert eta0[0] < 1e-15


def test_dsposv_diagonal_closed_form(oracle):
    # well-scaled diagonal: the binary32 solve misses tol, refinement reaches b/d
    d = np.array([1.0, 2.0, 3.0, 1.5, 4.0])
    b = np.array([1.0, -2.0, 3.0, 0.5, 7.0])
    x, it, info = oracle.dsposv(colmajor(np.diag(d)), b)
    assert info[0] == 0 and it[0] >= 1
    # stopping rule eta <= 1e-12 bounds the relative error by about cond * eta
    np.testing.assert_allclose(x[0], b / d, rtol=4 * 4.0 * 1e-12)
    # badly scaled diagonal: the normwise backward error of the binary32 solve is
    # already below tol, so the stopping rule accepts it without refinement
    d2 = np.array([1.0, 10.0, 1e3, 1e5, 1e6])
    x2, it2, _ = oracle.dsposv(colmajor(np.diag(d2)), b)
    assert it2[0] == 0
    assert oracle.backward_error(colmajor(np.diag(d2)), x2[0], b)[0] <= 1e-12
    np.testing.assert_allclose(x2[0], b / d2, rtol=1e-7)


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6])
def test_dsposv_backward_error(oracle, kappa):
    rng = np.random.default_rng(int(math.log10(kappa)))
    n = 48
    Z = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    Q = Q * np.sign(np.diag(R))
    s = kappa ** (-np.arange(n) / (n - 1))
    A = (Q * s) @ Q.T
    A = 0.5 * (A + A.T)
    b = rng.standard_normal(n)
    x, it, info = oracle.dsposv(colmajor(A), b, tol=1e-12, itmax=30)
    assert info[0] == 0 and it[0] >= 0
    eta = oracle.backward_error(colmajor(A), x[0], b)
    assert eta[0] <= 1e-12
    x64 = np.linalg.solve(A, b)
    assert np.abs(x[0] - x64).max() / np.abs(x64).max() < kappa * 1e-12 * 10


def test_dsposv_iterations_grow_with_condition(oracle):
    rng = np.random.default_rng(5)
    n = 32
    its = []
    for kappa in (1e1, 1e5):
        Q, R = np.linalg.qr(rng.standard_normal((n, n)))
        A = (Q * kappa ** (-np.arange(n) / (n - 1))) @ Q.T
        A = 0.5 * (A + A.T)
        _, it, _ = oracle.dsposv(colmajor(A), rng.standard_normal(n))
        its.append(it[0])
    assert its[0] <= its[1]
    assert its[1] >= 1


def test_dsposv_fallback_when_single_fails(oracle):
    # SPD in binary64 (eigenvalues 2e-9 and 2) but singular once rounded to binary32
    A = np.array([[1.0, 1.0 - 2e-9], [1.0 - 2e-9, 1.0]])
    b = np.array([1.0, 2.0])
    x, it, info = oracle.dsposv(colmajor(A), b)
    assert it[0] == -1 and info[0] == 0
    np.testing.assert_allclose(A @ x[0], b, atol=1e-6)
    assert oracle.backward_error(colmajor(A), x[0], b)[0] < 1e-14


def test_pivot_sqrt_double_rounding_is_innocuous():
    # The binary32 factorisation takes each pivot's square root in binary64 and rounds it to
    # binary32; the kernel takes the correctly rounded binary32 square root instead.  The two
    # agree for every positive binary32 d: sqrt(4^k d) = 2^k sqrt(d) exactly, so the mantissas
    # of [1, 4) (both exponent parities) cover every case.  Checked exhaustively here.
    lo = np.float32(1.0).view(np.uint32)
    hi = np.float32(4.0).view(np.uint32)
    for start in range(int(lo), int(hi), 1 << 22):
        d = np.arange(start, min(start + (1 << 22), int(hi)), dtype=np.uint32).view(np.float32)
        twice = np.sqrt(d.astype(np.float64)).astype(np.float32)
        once = np.sqrt(d)
        assert np.array_equal(twice.view(np.uint32), once.view(np.uint32))
    # the scaling argument, spot-checked at the ends of the range (subnormal and huge pivots)
    rng = np.random.default_rng(3)
    bits = rng.integers(1, 0x7F800000, size=1 << 20, dtype=np.uint32)
    d = bits.view(np.float32)
    assert np.array_equal(np.sqrt(d.astype(np.float64)).astype(np.float32).view(np.uint32),
                          np.sqrt(d).view(np.uint32))


def _chol_loss(oracle, A, Lbar):
    L, info = oracle.dpotrf_l(colmajor(A))
    assert info[0] == 0
    return float(np.sum(np.tril(L[0, :, :A.shape[0]].T) * Lbar))


@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_chol_adjoint_finite_differences(oracle, n):
    rng = np.random.default_rng(100 + n)
    G = rng.standard_normal((n, n))
    A = G @ G.T + n * np.eye(n)
    Lbar = np.tril(rng.standard_normal((n, n)))
    L, _ = oracle.dpotrf_l(colmajor(A))
    Abar = oracle.dpotrf_l_adjoint(L[0], Lbar.T.copy())  # column-major (ncols, ld)
    Abar_rm = Abar.T  # row-major (i, j)
    h = 1e-6
    for i in range(n):
        for j in range(i + 1):
            Ap, Am = A.copy(), A.copy()
            Ap[i, j] += h
            Am[i, j] -= h  # only the lower entry is read by the factorisation
            fd = (_chol_loss(oracle, Ap, Lbar) - _chol_loss(oracle, Am, Lbar)) / (2 * h)
            assert Abar_rm[i, j] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    assert np.all(np.triu(Abar_rm, 1) == 0)


def test_chol_adjoint_scalar(oracle):
    a = 2.25
    Abar = oracle.dpotrf_l_adjoint(np.array([[math.sqrt(a)]]), np.array([[1.0]]))
    assert Abar[0, 0] == pytest.approx(1.0 / (2.0 * math.sqrt(a)), rel=1e-15)


def test_chol_adjoint_matches_murray_form(oracle):
    """Symmetric gradient G = Phi-form of I. Murray (2016), evaluated with numpy:
    P = Phi(L^T Lbar) (lower triangle, halved diagonal), G = (S + S^T)/2 with
    S = L^{-T} P L^{-1}.  The oracle's lower-triangular result relates to G by
    G_ii = Abar_ii and G_ij = Abar_ij / 2 (i > j)."""
    rng = np.random.default_rng(77)
    n = 7
    Gm = rng.standard_normal((n, n))
    A = Gm @ Gm.T + n * np.eye(n)
    Lbar = np.tril(rng.standard_normal((n, n)))
    L = np.linalg.cholesky(A)
    P = np.tril(L.T @ Lbar)
    P[np.diag_indices(n)] *= 0.5
    Linv = np.linalg.inv(L)
    S = Linv.T @ P @ Linv
    Gsym = 0.5 * (S + S.T)
    Lc = colmajor(L)[0]
    Abar = oracle.dpotrf_l_adjoint(Lc, Lbar.T.copy()).T
    G_from_oracle = np.tril(Abar, -1) / 2
    G_from_oracle = G_from_oracle + G_from_oracle.T + np.diag(np.diag(Abar))
    np.testing.assert_allclose(G_from_oracle, Gsym, rtol=1e-10, atol=1e-12)


def _loss(oracle, Qd, J, B, W):
    out = oracle.spd_solve_loss_grad(Qd[None], J[None], B[None], W[None])
    return float(out["loss"][0])


def test_spd_solve_grad_finite_differences(oracle):
    rng = np.random.default_rng(123)
    n, q, r = 6, 3, 2
    Qd = 1 + rng.random(n)
    J = rng.standard_normal((q, n))  # column-major (ncols=q, ld=n)
    B = rng.standard_normal((r, n))
    W = rng.standard_normal((r, n))
    g = oracle.spd_solve_loss_grad(Qd[None], J[None], B[None], W[None])
    assert g["info"][0] == 0
    h = 1e-6
    for name, X, G in (("J", J, g["Jbar"][0]), ("Q", Qd, g["Qbar"][0]), ("B", B, g["Bbar"][0]),
                       ("W", W, g["Wbar"][0])):
        for idx in np.ndindex(X.shape):
            Xp, Xm = X.copy(), X.copy()
            Xp[idx] += h
            Xm[idx] -= h
            args_p = dict(Qd=Qd, J=J, B=B, W=W)
            args_m = dict(Qd=Qd, J=J, B=B, W=W)
            key = {"J": "J", "Q": "Qd", "B": "B", "W": "W"}[name]
            args_p[key], args_m[key] = Xp, Xm
            fd = (_loss(oracle, **args_p) - _loss(oracle, **args_m)) / (2 * h)
            assert G[idx] == pytest.approx(fd, rel=1e-6, abs=1e-8), (name, idx)
