"""torch.autograd Functions whose forward and backward run in this library's kernels.

Tensors are batches of column-major matrices, shape (batch, ncols, ld), as in
the rest of the binding.  Each Function calls the C ABI forward routine and,
on the backward pass, the matching hand-written adjoint routine:

  Gemm          C = alpha op(A) op(B) + beta C0   -> bf_dgemm_backward_strided_batched
  TriSolve      op(A) X = alpha B / X op(A) = alpha B -> bf_dtrsm_backward_strided_batched
  CholSolve     X = L^{-T} L^{-1} B (dpotrs)      -> bf_dpotrs_backward_strided_batched
  Cholesky      A = L L^T (lower)                 -> bf_dpotrf_backward_strided_batched
  SyrkCholesky  L = chol(C0 + A A^T), the fused dsyrk + dpotrf routine (section 5)
                                                  -> bf_dpotrf_backward_strided_batched, then
                                                     one dgemm

Cholesky's gradient is the symmetric one (the input is treated as a
symmetric matrix, as the factorisation reads only its lower triangle).
`spd_solve_loss` chains them into the differentiation workload
loss = sum((Q + J J^T)^{-1} B .* W).
"""
from __future__ import annotations

import torch

from . import (_batch_dims, _ch, _check, _ptr, _stream, bf_dgemm_backward_strided_batched,
               bf_dpotrf_backward_strided_batched, bf_dpotrs_backward_strided_batched,
               bf_dtrsm_backward_strided_batched, dgemm, dpotrf, dsyrk_dpotrf, dtrfill, dtrsm)


def _same_batch(names, *Xs):
    """The adjoints write one gradient matrix per problem, so every operand must hold one matrix
    per problem: a matrix shared by the whole batch (batch count 1) would need its per-problem
    gradients summed, which these Functions do not do.  Expand such an operand first."""
    counts = [X.shape[0] for X in Xs]
    if any(c != counts[0] for c in counts):
        raise ValueError("differentiable operands must hold one matrix per problem; got batch counts "
                         + ", ".join(f"{nm}={c}" for nm, c in zip(names, counts)))


def _out_like(X, rows, cols):
    """A gradient buffer shaped like X (..., ncols, ld) of which the adjoint kernel writes the
    leading rows x cols block of every problem in full: uninitialised when that block is all of
    X, zeroed when X has padding rows or columns beyond it."""
    return torch.empty_like(X) if (X.shape[-1], X.shape[-2]) == (rows, cols) else torch.zeros_like(X)


class Gemm(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, C0, transa, transb, alpha, beta, m, n, k):
        _same_batch("ABC", A, B, C0)
        C = C0.clone(memory_format=torch.contiguous_format)
        dgemm(transa, transb, alpha, A, B, beta, C, m=m, n=n, k=k)
        ctx.save_for_backward(A, B)
        ctx.args = (transa, transb, alpha, beta, m, n, k)
        return C

    @staticmethod
    def backward(ctx, Cbar):
        A, B = ctx.saved_tensors
        transa, transb, alpha, beta, m, n, k = ctx.args
        Cbar = Cbar.contiguous()
        need_a, need_b, need_c = ctx.needs_input_grad[:3]
        ta, tb = transa in "Tt", transb in "Tt"
        Abar = _out_like(A, k if ta else m, m if ta else k) if need_a else None
        Bbar = _out_like(B, n if tb else k, k if tb else n) if need_b else None
        C0bar = _out_like(Cbar, m, n) if need_c else None
        bA, cA, ldA, sA = _batch_dims(A)
        bB, cB, ldB, sB = _batch_dims(B)
        bC, cC, ldC, sC = _batch_dims(Cbar)

        def opt(t):
            if t is None:
                return None, 1, 0
            _, _, ld, st = _batch_dims(t)
            return _ptr(t), ld, st

        pa, lda_, sa = opt(Abar)
        pb, ldb_, sb = opt(Bbar)
        pc, ldc_, sc = opt(C0bar)
        _check("bf_dgemm_backward_strided_batched", bf_dgemm_backward_strided_batched(
            _ch(transa), _ch(transb), m, n, k, alpha, _ptr(A), ldA, sA if bA > 1 else 0, _ptr(B), ldB,
            sB if bB > 1 else 0, beta, _ptr(Cbar), ldC, sC, pa, max(lda_, ldA) if pa else ldA, sa, pb,
            max(ldb_, ldB) if pb else ldB, sb, pc, max(ldc_, ldC) if pc else ldC, sc, bC, _stream()))
        return Abar, Bbar, C0bar, None, None, None, None, None, None, None


class TriSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, side, uplo, transa, diag, alpha, m, n):
        _same_batch("AB", A, B)
        X = B.clone(memory_format=torch.contiguous_format)
        dtrsm(side, uplo, transa, diag, alpha, A, X, m=m, n=n)
        ctx.save_for_backward(A, X)
        ctx.args = (side, uplo, transa, diag, alpha, m, n)
        return X

    @staticmethod
    def backward(ctx, Xbar):
        A, X = ctx.saved_tensors
        side, uplo, transa, diag, alpha, m, n = ctx.args
        Z = Xbar.clone(memory_format=torch.contiguous_format)
        Abar = torch.zeros_like(A) if ctx.needs_input_grad[0] else None
        bA, cA, ldA, sA = _batch_dims(A)
        bX, cX, ldX, sX = _batch_dims(X)
        bZ, cZ, ldZ, sZ = _batch_dims(Z)
        _check("bf_dtrsm_backward_strided_batched", bf_dtrsm_backward_strided_batched(
            _ch(side), _ch(uplo), _ch(transa), _ch(diag), m, n, alpha, _ptr(A), ldA, sA if bA > 1 else 0,
            _ptr(X), ldX, sX, _ptr(Z), ldZ, sZ, _ptr(Abar) if Abar is not None else None, ldA,
            sA if Abar is not None else 0, bX, _stream()))
        return Abar, Z, None, None, None, None, None, None, None


class CholSolve(torch.autograd.Function):
    """X = L^{-T} L^{-1} B from a lower factor L (A = L L^T; 'U': X = U^{-1} U^{-T} B), B n x nrhs.

    The same two solves as TriSolve("L", "N") then TriSolve("L", "T"), but one backward call
    gives both solves' adjoints, with the factor's gradient summed in its own buffer instead of
    by autograd, and B's gradient in place of a copy of Xbar."""

    @staticmethod
    def forward(ctx, L, B, uplo, n, nrhs):
        _same_batch("LB", L, B)
        up = uplo in "Uu"
        Y = B.clone(memory_format=torch.contiguous_format)
        dtrsm("L", uplo, "T" if up else "N", "N", 1.0, L, Y, m=n, n=nrhs)
        X = Y.clone()
        dtrsm("L", uplo, "N" if up else "T", "N", 1.0, L, X, m=n, n=nrhs)
        ctx.save_for_backward(L, X, Y)
        ctx.args = (uplo, n, nrhs)
        return X

    @staticmethod
    def backward(ctx, Xbar):
        L, X, Y = ctx.saved_tensors
        uplo, n, nrhs = ctx.args
        Z = Xbar.clone(memory_format=torch.contiguous_format)  # becomes Bbar
        Lbar = _out_like(L, n, n)  # all n x n are written (zeros off the triangle)
        bL, cL, ldL, sL = _batch_dims(L)
        bX, cX, ldX, sX = _batch_dims(X)
        bY, cY, ldY, sY = _batch_dims(Y)
        bZ, cZ, ldZ, sZ = _batch_dims(Z)
        _check("bf_dpotrs_backward_strided_batched", bf_dpotrs_backward_strided_batched(
            _ch(uplo), n, nrhs, _ptr(L), ldL, sL, _ptr(X), ldX, sX, _ptr(Y), ldY, sY, _ptr(Z), ldZ, sZ,
            _ptr(Lbar), ldL, sL, bL, _stream()))
        return Lbar, (Z if ctx.needs_input_grad[1] else None), None, None, None


class Cholesky(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, n):
        L = A.clone(memory_format=torch.contiguous_format)
        info = dpotrf(L, n=n)
        # strict upper triangle zeroed; a problem that is not positive definite becomes NaN, so
        # that its gradient is NaN too instead of a finite but meaningless value
        dtrfill(L, info, n=n)
        ctx.save_for_backward(L)
        ctx.n = n
        ctx.info = info
        return L

    @staticmethod
    def backward(ctx, Lbar):
        (L,) = ctx.saved_tensors
        return _cholesky_adjoint(L, Lbar, ctx.n), None


def _cholesky_adjoint(L, Lbar, n):
    """The symmetric gradient of A = L L^T with respect to A (full, symmetric) from Lbar."""
    Lbar = Lbar.contiguous()
    Abar = _out_like(L, n, n)  # the kernels write all n x n of every problem
    bL, cL, ldL, sL = _batch_dims(L)
    bB, cB, ldB, sB = _batch_dims(Lbar)
    _check("bf_dpotrf_backward_strided_batched", bf_dpotrf_backward_strided_batched(
        _ch("L"), n, _ptr(L), ldL, sL, _ptr(Lbar), ldB, sB, _ptr(Abar), ldL, sL, bL, _stream()))
    return Abar


class SyrkCholesky(torch.autograd.Function):
    """L = chol(C0 + A A^T) (lower; A n x k), forward by the fused dsyrk + dpotrf routine.

    The Cholesky adjoint gives the symmetric C = C0 + A A^T its gradient Cbar (symmetric), so
    Abar = (Cbar + Cbar^T) A = 2 Cbar A takes one dgemm, and C0bar = Cbar.  Against a general
    product A B^T with A = B (Gemm), that is one dgemm and one sum fewer in the backward, and
    half the forward product (only the lower triangle of A A^T is formed)."""

    @staticmethod
    def forward(ctx, A, C0, n, k):
        _same_batch("AC", A, C0)
        L = C0.clone(memory_format=torch.contiguous_format)
        info = dsyrk_dpotrf(A, L, n=n, k=k)
        # strict upper triangle zeroed; a problem that is not positive definite becomes NaN
        dtrfill(L, info, n=n)
        ctx.save_for_backward(A, L)
        ctx.nk = (n, k)
        return L

    @staticmethod
    def backward(ctx, Lbar):
        A, L = ctx.saved_tensors
        n, k = ctx.nk
        Cbar = _cholesky_adjoint(L, Lbar, n)
        Abar = None
        if ctx.needs_input_grad[0]:
            Abar = _out_like(A, n, k)
            dgemm("N", "N", 2.0, Cbar, A, 0.0, Abar, m=n, n=k, k=n)
        return Abar, (Cbar if ctx.needs_input_grad[1] else None), None, None


def spd_solve_loss(Qd, J, B, W):
    """loss = sum(X .* W), X = L^{-T} L^{-1} B, L = chol(Q + J J^T), Q = diag(Qd).

    Qd (batch, n); J (batch, q, n); B, W (batch, r, n) -- column-major, ld = n.
    Returns (loss, X, L).
    """
    batch, n = Qd.shape
    q, r = J.shape[1], B.shape[1]
    C0 = torch.diag_embed(Qd)  # symmetric: the (ncols, ld) layout is the same
    L = SyrkCholesky.apply(J, C0, n, q)
    X = CholSolve.apply(L, B, "L", n, r)
    return (X * W).sum(), X, L
