"""GPU parity of the hand-written backward kernels and the autograd chain.

* dgemm adjoint: against the oracle's dgemm applied to the adjoint formulas;
* dtrsm adjoint (all 16 cases): against central finite differences of the
  oracle's forward solve (an independent route), and the formula;
* Cholesky adjoint: against the oracle's reverse mode of its own unblocked
  loop (converted between the symmetric and lower-triangular conventions);
* the differentiation workload loss = sum((Q + J J^T)^{-1} B .* W): autograd
  gradient of the GPU chain against the oracle's closed-form gradient and
  against central finite differences (h = 1e-6) of the GPU forward pass,
  relative error <= 1e-8 (both).
"""
import contextlib
import itertools

import numpy as np
import pytest
import torch

import bfsynth
from bfhelp import forced, gpu, host, normwise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from bfhelp import build_lib
    return build_lib()


@pytest.fixture(scope="module")
def ag(bf):
    from paper_1902_08115_gb300 import autograd
    return autograd


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
@pytest.mark.parametrize("m,n,k", [(5, 7, 3), (24, 24, 24), (33, 17, 40)])
def test_dgemm_backward(bf, ag, oracle, ta, tb, m, n, k):
    batch, alpha, beta = 6, 0.75, -1.5
    rA, cA = (m, k) if ta == "N" else (k, m)
    rB, cB = (k, n) if tb == "N" else (n, k)
    A = bfsynth.randn_batch(batch, rA, cA, rA, 1).numpy()
    B = bfsynth.randn_batch(batch, rB, cB, rB, 2).numpy()
    C0 = bfsynth.randn_batch(batch, m, n, m, 3).numpy()
    Cb = bfsynth.randn_batch(batch, m, n, m, 4).numpy()
    At, Bt, Ct = (gpu(x).requires_grad_(True) for x in (A, B, C0))
    C = ag.Gemm.apply(At, Bt, Ct, ta, tb, alpha, beta, m, n, k)
    C.backward(gpu(Cb))
    # references from the adjoint formulas, evaluated with the oracle's dgemm
    Z = lambda r, c: np.zeros((batch, c, r))
    if ta == "N":
        refA = oracle.dgemm("N", "T" if tb == "N" else "N", m, k, n, alpha, Cb, B, 0.0, Z(m, k))
    else:
        refA = oracle.dgemm(tb, "T", k, m, n, alpha, B, Cb, 0.0, Z(k, m))
    if tb == "N":
        refB = oracle.dgemm("T" if ta == "N" else "N", "N", k, n, m, alpha, A, Cb, 0.0, Z(k, n))
    else:
        refB = oracle.dgemm("T", ta, n, k, m, alpha, Cb, A, 0.0, Z(n, k))
    assert normwise(host(At.grad), refA, rA) <= 1e-13
    assert normwise(host(Bt.grad), refB, rB) <= 1e-13
    assert normwise(host(Ct.grad), beta * Cb, m) <= 1e-15


def tri(batch, order, uplo, diag, seed):
    g = np.random.default_rng(seed)
    T = g.standard_normal((batch, order, order)) / np.sqrt(order)
    T = np.tril(T) if uplo == "L" else np.triu(T)
    d = 1.5 + g.random((batch, order))
    for q in range(batch):
        np.fill_diagonal(T[q], 1.0 if diag == "U" else d[q])
    return np.ascontiguousarray(np.transpose(T, (0, 2, 1)))  # column-major


@pytest.mark.parametrize("side,uplo,ta,diag", list(itertools.product("LR", "LU", "NT", "NU")))
def test_dtrsm_backward(bf, ag, oracle, side, uplo, ta, diag):
    check_dtrsm_backward(ag, oracle, side, uplo, ta, diag, 5, 4)


@pytest.mark.parametrize("side,uplo,ta,diag", list(itertools.product("LR", "LU", "NT", "NU")))
def test_dtrsm_backward_tiny_product(bf, ag, oracle, side, uplo, ta, diag):
    """Orders and right-hand sides <= 4 with the one-thread-per-problem dgemm forced: the
    adjoint's product is kept on the stored triangle there too (that kernel itself stores every
    entry of its result)."""
    with forced(bf, bf.ROUTINE_DGEMM, -1, bf.VARIANT_TINY):
        check_dtrsm_backward(ag, oracle, side, uplo, ta, diag, 3, 4)
        check_dtrsm_backward(ag, oracle, side, uplo, ta, diag, 4, 3)


def check_dtrsm_backward(ag, oracle, side, uplo, ta, diag, m, n):
    batch, alpha = 3, 1.25
    order = m if side == "L" else n
    A = tri(batch, order, uplo, diag, 7)
    B = bfsynth.randn_batch(batch, m, n, m, 8).numpy()
    W = bfsynth.randn_batch(batch, m, n, m, 9).numpy()
    At, Bt = gpu(A).requires_grad_(True), gpu(B).requires_grad_(True)
    X = ag.TriSolve.apply(At, Bt, side, uplo, ta, diag, alpha, m, n)
    (X * gpu(W)).sum().backward()
    gA, gB = host(At.grad), host(Bt.grad)

    def loss(Am, Bm):
        return float(np.sum(oracle.dtrsm(side, uplo, ta, diag, m, n, alpha, Am, Bm) * W))

    h = 1e-6
    fdB = np.zeros_like(B)
    for idx in np.ndindex(B.shape):
        Bp, Bm = B.copy(), B.copy()
        Bp[idx] += h
        Bm[idx] -= h
        fdB[idx] = (loss(A, Bp) - loss(A, Bm)) / (2 * h)
    assert rel(gB, fdB) <= 1e-8
    fdA = np.zeros_like(A)
    for q in range(batch):
        for j in range(order):
            for i in range(order):
                stored = (i >= j) if uplo == "L" else (i <= j)
                if not stored or (diag == "U" and i == j):
                    continue
                Ap, Am = A.copy(), A.copy()
                Ap[q, j, i] += h
                Am[q, j, i] -= h
                fdA[q, j, i] = (loss(Ap, B) - loss(Am, B)) / (2 * h)
    assert rel(gA, fdA) <= 1e-8


@pytest.mark.parametrize("n", [1, 2, 5, 16, 32, 33])
def test_dpotrf_backward(bf, ag, oracle, n):
    batch = 5
    S = bfsynth.spd_batch(batch, n, n, 10 + n).numpy()
    Lb = np.ascontiguousarray(np.triu(bfsynth.randn_batch(batch, n, n, n, 11).numpy()))  # lower in (j, i)
    St = gpu(S).requires_grad_(True)
    L = ag.Cholesky.apply(St, n)
    L.backward(gpu(Lb))
    G = host(St.grad)  # symmetric gradient, column-major
    Lo, _ = oracle.dpotrf_l(S)
    for q in range(batch):
        ref = oracle.dpotrf_l_adjoint(Lo[q], Lb[q])  # lower-triangular convention, (ncols, ld)
        Gq = G[q]
        # tril convention: Abar_ij = 2 G_ij (i > j), Abar_ii = G_ii
        conv = np.where(np.arange(n)[None, :] > np.arange(n)[:, None], 2 * Gq, 0.0)  # [j, i], i > j
        conv = conv + np.diag(np.diag(Gq))
        assert rel(conv, ref) <= 1e-12
        assert rel(Gq, Gq.T) <= 1e-15


def test_spd_solve_gradient(bf, ag, oracle):
    """The differentiation workload (n = 32, J 32x16, B and W 32x8) at a reduced batch."""
    batch, n, q, r = 256, 32, 16, 8
    Qd, J, B, W = (x.numpy() for x in bfsynth.diff_batch(batch, n, q, r, seed=bfsynth.BASE_SEED))
    ts = [gpu(x).requires_grad_(True) for x in (Qd, J, B, W)]
    loss, X, L = ag.spd_solve_loss(*ts)
    loss.backward()
    g = [host(t.grad) for t in ts]
    ref = oracle.spd_solve_loss_grad(Qd, J, B, W)
    assert (ref["info"] == 0).all()
    assert rel(host(X.detach()), ref["X"]) <= 1e-12
    for got, key in zip(g, ("Qbar", "Jbar", "Bbar", "Wbar")):
        assert rel(got, ref[key]) <= 1e-8, key
    # central finite differences of the GPU forward pass, per-problem losses
    h = 1e-6
    rng = np.random.default_rng(0)
    fd, an = [], []
    base = [x.copy() for x in (Qd, J, B, W)]
    for which in range(4):
        for _ in range(6):
            prob = int(rng.integers(batch))
            idx = tuple(int(rng.integers(s)) for s in base[which].shape[1:])
            vals = []
            for sgn in (1, -1):
                xs = [x.copy() for x in base]
                xs[which][(prob,) + idx] += sgn * h
                with torch.no_grad():
                    _, Xp, _ = ag.spd_solve_loss(*(gpu(x) for x in xs))
                vals.append(float(np.sum(host(Xp[prob]) * xs[3][prob])))
            fd.append((vals[0] - vals[1]) / (2 * h))
            an.append(g[which][(prob,) + idx])
    assert rel(an, fd) <= 1e-8, (an, fd)


@pytest.mark.parametrize("uplo", "LU")
@pytest.mark.parametrize("n,r,tiny", [(1, 1, False), (3, 4, True), (5, 3, False), (32, 8, False),
                                      (33, 4, False), (70, 2, False)])
def test_cholsolve_matches_trisolve_chain(bf, ag, oracle, uplo, n, r, tiny):
    """CholSolve (both solves' adjoints in one call, the factor's gradient summed in one buffer)
    against the chain of two TriSolve Functions with autograd's sum: the same solution, Bbar and
    Lbar within rounding, zeros in the factor gradient's other strict triangle; and the
    factor gradient's stored triangle against central differences of the oracle's solves."""
    batch = 6
    L = tri(batch, n, uplo, "N", 11 + n)
    B = bfsynth.randn_batch(batch, n, r, n, 12).numpy()
    W = bfsynth.randn_batch(batch, n, r, n, 13).numpy()
    t1, t2 = ("T", "N") if uplo == "U" else ("N", "T")
    outs = []
    ctx = forced(bf, bf.ROUTINE_DGEMM, -1, bf.VARIANT_TINY) if tiny else contextlib.nullcontext()
    with ctx:
        for fused in (True, False):
            Lt, Bt = gpu(L).requires_grad_(True), gpu(B).requires_grad_(True)
            if fused:
                X = ag.CholSolve.apply(Lt, Bt, uplo, n, r)
            else:
                Y = ag.TriSolve.apply(Lt, Bt, "L", uplo, t1, "N", 1.0, n, r)
                X = ag.TriSolve.apply(Lt, Y, "L", uplo, t2, "N", 1.0, n, r)
            (X * gpu(W)).sum().backward()
            outs.append((host(X.detach()), host(Lt.grad), host(Bt.grad)))
    (Xf, gLf, gBf), (Xc, gLc, gBc) = outs
    assert np.array_equal(Xf, Xc)
    assert rel(gBf, gBc) <= 1e-14
    assert rel(gLf, gLc) <= 1e-13
    # column-major storage: [q, j, i] is entry (i, j), so the strict upper triangle (i < j) is
    # the array's strict lower one
    other = (np.tril(np.ones((n, n)), -1) if uplo == "L" else np.triu(np.ones((n, n)), 1)).astype(bool)
    for q in range(batch):
        assert np.all(gLf[q][other] == 0.0)
    if n <= 5:
        h = 1e-6

        def loss(Lm):
            Y = oracle.dtrsm("L", uplo, t1, "N", n, r, 1.0, Lm, B)
            return float(np.sum(oracle.dtrsm("L", uplo, t2, "N", n, r, 1.0, Lm, Y) * W))

        fd = np.zeros_like(L)
        for q in range(batch):
            for j in range(n):
                for i in range(n):
                    if (i >= j) if uplo == "L" else (i <= j):
                        Lp, Lm = L.copy(), L.copy()
                        Lp[q, j, i] += h
                        Lm[q, j, i] -= h
                        fd[q, j, i] = (loss(Lp) - loss(Lm)) / (2 * h)
        assert rel(gLf, fd) <= 1e-8


def test_syrk_cholesky_matches_gemm_chain(bf, ag):
    """The fused Function L = chol(C0 + A A^T) (forward by the fused dsyrk + dpotrf routine,
    Abar = 2 Cbar A) gives the gradients of the general chain Gemm(A, A^T) -> Cholesky: the same
    factor, and Abar, C0bar within rounding, for a downstream loss of every entry of L."""
    batch, n, k = 64, 20, 7
    g = np.random.default_rng(5)
    A = g.standard_normal((batch, k, n))
    C0 = np.zeros((batch, n, n))
    for q in range(batch):
        C0[q] += np.diag(1.0 + g.random(n)) * n
    Lw = g.standard_normal((batch, n, n))
    outs = []
    for fused in (True, False):
        At, Ct = gpu(A).requires_grad_(True), gpu(C0).requires_grad_(True)
        if fused:
            L = ag.SyrkCholesky.apply(At, Ct, n, k)
        else:
            L = ag.Cholesky.apply(ag.Gemm.apply(At, At, Ct, "N", "T", 1.0, 1.0, n, n, k), n)
        (L * gpu(np.tril(Lw.transpose(0, 2, 1)).transpose(0, 2, 1))).sum().backward()
        outs.append((host(L.detach()), host(At.grad), host(Ct.grad)))
    assert rel(outs[0][0], outs[1][0]) <= 1e-13
    assert rel(outs[0][1], outs[1][1]) <= 1e-12
    assert rel(outs[0][2], outs[1][2]) <= 1e-12


def test_cholesky_failure_poisons_factor_and_gradient(bf, ag):
    """A problem that is not positive definite comes out of the forward pass as NaN, so its
    gradient is NaN as well; the other problems of the batch keep finite, unchanged results."""
    batch, n, bad = 6, 9, 2
    S = bfsynth.spd_batch(batch, n, n, 31).numpy()
    S[bad, 4, 4] = -1.0  # leading minor 5 is not positive
    Lb = np.ascontiguousarray(np.triu(bfsynth.randn_batch(batch, n, n, n, 32).numpy()))
    St = gpu(S).requires_grad_(True)
    L = ag.Cholesky.apply(St, n)
    L.backward(gpu(Lb))
    Lh, G = host(L.detach()), host(St.grad)
    assert np.isnan(Lh[bad]).all()
    assert np.isnan(G[bad]).all()
    ok = [q for q in range(batch) if q != bad]
    assert np.isfinite(Lh[ok]).all() and np.isfinite(G[ok]).all()
    # strict upper triangle of every good factor is zero, (j, i) layout: i < j
    for q in ok:
        assert not np.triu(Lh[q].T, 1).any()
    # the good problems are the same as in a batch without the failing one
    St2 = gpu(S[ok]).requires_grad_(True)
    L2 = ag.Cholesky.apply(St2, n)
    L2.backward(gpu(Lb[ok]))
    assert normwise(host(L2.detach()), Lh[ok], n) <= 1e-13
    assert rel(host(St2.grad), G[ok]) <= 1e-13


@pytest.mark.parametrize("n", [1, 5, 32, 33])
def test_dpotrf_backward_upper(bf, oracle, n):
    """uplo 'U' of the Cholesky adjoint through the C ABI: A = U^T U with U and Ubar in upper
    triangles; the symmetric gradient must equal the lower one of L = U^T, Lbar = Ubar^T (the
    oracle's reverse mode, converted as in test_dpotrf_backward)."""
    import ctypes
    batch = 4
    S = bfsynth.spd_batch(batch, n, n, 40 + n).numpy()
    Uo, info = oracle.dpotrf_u(S, n=n)
    assert (info == 0).all()
    Ub = np.ascontiguousarray(np.tril(bfsynth.randn_batch(batch, n, n, n, 41).numpy()))  # upper in (j, i)
    Ug, Ubg = gpu(Uo), gpu(Ub)
    G = torch.zeros(batch, n, n, dtype=torch.float64, device="cuda")
    vp = ctypes.c_void_p
    r = bf.bf_dpotrf_backward_strided_batched(b"U", n, vp(Ug.data_ptr()), n, n * n, vp(Ubg.data_ptr()), n, n * n,
                                              vp(G.data_ptr()), n, n * n, batch, bf._stream())
    assert r == 0
    G = host(G)
    for q in range(batch):
        L = np.ascontiguousarray(Uo[q].T)      # lower factor, (ncols, ld) layout
        Lb = np.ascontiguousarray(Ub[q].T)     # its adjoint, lower
        ref = oracle.dpotrf_l_adjoint(L, Lb)
        Gq = G[q]
        conv = np.where(np.arange(n)[None, :] > np.arange(n)[:, None], 2 * Gq, 0.0) + np.diag(np.diag(Gq))
        assert rel(conv, ref) <= 1e-12
        assert rel(Gq, Gq.T) <= 1e-15
