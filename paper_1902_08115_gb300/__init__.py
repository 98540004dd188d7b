"""Batched small-matrix FP64 BLAS/LAPACK for one GB300 (sm_103a).

Thin Python binding of the C ABI in include/bfgpu.h: argument marshalling
only.  Every step of every routine runs in the library's CUDA kernels
(libbfgpu.so); there is no CPU fallback, and importing this package fails
loudly when the compiled library is missing.

Tensor convention: a batch of column-major matrices with ``ncols`` columns and
leading dimension ``ld`` is a contiguous float64 CUDA tensor of shape
``(batch, ncols, ld)``; element (i, j) of problem b is ``X[b, j, i]`` (the
BLAS storage the paper keeps, section 2.1).  Work is enqueued on torch's
current CUDA stream.

The functions with a ``bf_`` prefix are the raw C entry points (ctypes
functions taking device pointers); the lower-case helpers take tensors.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libbfgpu.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python paper_1902_08115_gb300/build.py); there is no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

_c = ctypes.c_char
_i = ctypes.c_int
_ll = ctypes.c_longlong
_d = ctypes.c_double
_vp = ctypes.c_void_p
_ip = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "bf_dgemm": [_c, _c, _i, _i, _i, _d, _vp, _i, _vp, _i, _d, _vp, _i, _vp],
    "bf_dgemm_strided_batched": [_c, _c, _i, _i, _i, _d, _vp, _i, _ll, _vp, _i, _ll, _d, _vp, _i, _ll,
                                 _i, _vp],
    "bf_dgemm_batched": [_c, _c, _i, _i, _i, _d, _vp, _i, _vp, _i, _d, _vp, _i, _i, _vp],
    "bf_dtrsm": [_c, _c, _c, _c, _i, _i, _d, _vp, _i, _vp, _i, _vp],
    "bf_dtrsm_strided_batched": [_c, _c, _c, _c, _i, _i, _d, _vp, _i, _ll, _vp, _i, _ll, _i, _vp],
    "bf_dtrsm_batched": [_c, _c, _c, _c, _i, _i, _d, _vp, _i, _vp, _i, _i, _vp],
    "bf_dpotrf": [_c, _i, _vp, _i, _vp, _vp],
    "bf_dpotrf_strided_batched": [_c, _i, _vp, _i, _ll, _vp, _i, _vp],
    "bf_dpotrf_batched": [_c, _i, _vp, _i, _vp, _i, _vp],
    "bf_dgemm_vbatched": [_c, _c, _vp, _vp, _vp, _d, _vp, _vp, _vp, _vp, _d, _vp, _vp, _i, _i, _i, _i, _vp,
                          _vp],
    "bf_dtrsm_vbatched": [_c, _c, _c, _c, _vp, _vp, _d, _vp, _vp, _vp, _vp, _i, _i, _i, _vp, _vp],
    "bf_dpotrf_vbatched": [_c, _vp, _vp, _vp, _vp, _i, _i, _vp],
    "bf_dpotrs": [_c, _i, _i, _vp, _i, _vp, _i, _vp],
    "bf_dpotrs_strided_batched": [_c, _i, _i, _vp, _i, _ll, _vp, _i, _ll, _i, _vp],
    "bf_dpotrs_batched": [_c, _i, _i, _vp, _i, _vp, _i, _i, _vp],
    "bf_dpotrs_vbatched": [_c, _vp, _vp, _vp, _vp, _vp, _vp, _i, _i, _i, _vp, _vp],
    "bf_tune_set": [_i, _i, _i, _i, _i, _i, _i, _i, _i],
    "bf_tune_set_batch_rule": [_i, _i, _i, _i, _ll, _ll, _ll],
    "bf_tune_clear": [],
    "bf_tune_query": [_i, _i, _i, _i, _i, _ll, _ip],
    "bf_status_string": [_i],
    "bf_dsposv_strided_batched": [_c, _i, _i, _vp, _i, _ll, _vp, _i, _ll, _vp, _i, _ll, _vp, _vp, _d, _i,
                                  _vp, ctypes.c_size_t, _i, _vp],
    "bf_dsposv_workspace_bytes": [_i, _i],
    "bf_dgemm_backward_strided_batched": [_c, _c, _i, _i, _i, _d, _vp, _i, _ll, _vp, _i, _ll, _d, _vp, _i,
                                          _ll, _vp, _i, _ll, _vp, _i, _ll, _vp, _i, _ll, _i, _vp],
    "bf_dtrsm_backward_strided_batched": [_c, _c, _c, _c, _i, _i, _d, _vp, _i, _ll, _vp, _i, _ll, _vp, _i,
                                          _ll, _vp, _i, _ll, _i, _vp],
    "bf_dpotrf_backward_strided_batched": [_c, _i, _vp, _i, _ll, _vp, _i, _ll, _vp, _i, _ll, _i, _vp],
    "bf_dpotrs_backward_strided_batched": [_c, _i, _i, _vp, _i, _ll, _vp, _i, _ll, _vp, _i, _ll, _vp, _i, _ll,
                                           _vp, _i, _ll, _i, _vp],
    "bf_dtrfill_strided_batched": [_c, _i, _vp, _i, _ll, _vp, _i, _vp],
    "bf_ragged_workspace_bytes": [_i],
    "bf_ragged_potrf_potrs_plan_create": [_i, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _i, _i,
                                          _vp, ctypes.POINTER(_vp)],
    "bf_ragged_plan_launch": [_vp, _vp],
    "bf_ragged_plan_info": [_vp, _ip],
    "bf_ragged_plan_destroy": [_vp],
    "bf_ragged_potrf_potrs_noalloc": [_i, _vp, _i, _vp, _vp, _vp, _vp, _vp, _i, _i, _vp],
    "bf_dsyrk": [_c, _c, _i, _i, _d, _vp, _i, _d, _vp, _i, _vp],
    "bf_dsyrk_strided_batched": [_c, _c, _i, _i, _d, _vp, _i, _ll, _d, _vp, _i, _ll, _i, _vp],
    "bf_dsyrk_batched": [_c, _c, _i, _i, _d, _vp, _i, _d, _vp, _i, _i, _vp],
    "bf_dsyrk_dpotrf": [_i, _i, _vp, _i, _vp, _i, _vp, _vp],
    "bf_dsyrk_dpotrf_strided_batched": [_i, _i, _vp, _i, _ll, _vp, _i, _ll, _vp, _i, _vp],
    "bf_dtrmm": [_c, _c, _c, _c, _i, _i, _d, _vp, _i, _vp, _i, _vp],
    "bf_dtrmm_strided_batched": [_c, _c, _c, _c, _i, _i, _d, _vp, _i, _ll, _vp, _i, _ll, _i, _vp],
    "bf_dtrmm_batched": [_c, _c, _c, _c, _i, _i, _d, _vp, _i, _vp, _i, _i, _vp],
    "bf_dgetrf": [_i, _i, _vp, _i, _vp, _vp, _vp],
    "bf_dgetrf_strided_batched": [_i, _i, _vp, _i, _ll, _vp, _ll, _vp, _i, _vp],
    "bf_dgetrs": [_c, _i, _i, _vp, _i, _vp, _vp, _i, _vp],
    "bf_dgetrs_strided_batched": [_c, _i, _i, _vp, _i, _ll, _vp, _ll, _vp, _i, _ll, _i, _vp],
    "bf_riccati_workspace_bytes": [_i, _i, _i],
    "bf_riccati_strided_batched": [_i, _i, _i, _vp, _ll, _vp, _ll, _vp, _ll, _vp, _ll, _vp, _i, _vp,
                                   ctypes.c_size_t, _i, _vp],
    "bf_launch_count": [],
    "bf_probe_fp64": [_i, _i, _vp, _vp],
    "bf_probe_fp64_ex": [_i, _i, _i, _i, _i, _vp, _vp],
    "bf_probe_kind": [_i, _i, _i, _i, _vp, _vp],
}
_RES = {"bf_tune_clear": None, "bf_status_string": ctypes.c_char_p, "bf_ragged_workspace_bytes": ctypes.c_size_t,
        "bf_dsposv_workspace_bytes": ctypes.c_size_t, "bf_riccati_workspace_bytes": ctypes.c_size_t,
        "bf_launch_count": ctypes.c_ulonglong}

for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _RES.get(_name, _i)
    globals()[_name] = _f

ROUTINE_DGEMM, ROUTINE_DTRSM, ROUTINE_DPOTRF, ROUTINE_DGETRF = 0, 1, 2, 3
VARIANT_DIRECT, VARIANT_PACKED, VARIANT_BLOCKED, VARIANT_TINY, VARIANT_CTA, VARIANT_TEAM = 0, 1, 2, 3, 4, 5
VARIANT_GROUP = 6
TUNE_FORCE = 0x100  # or into a variant: the table entry holds at every batch size
ERR_CUDA, ERR_NOT_SUPPORTED, ERR_NOALLOC_LIMIT = 1001, 1002, 1003
RAGGED_NOALLOC_MAX = 32768


class BFError(RuntimeError):
    """A library call returned a nonzero status."""

    def __init__(self, name: str, status: int):
        self.status = status
        msg = bf_status_string(status).decode()
        super().__init__(f"{name} returned {status}: {msg}")


def _check(name: str, status: int) -> None:
    if status != 0:
        raise BFError(name, status)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _ch(c: str) -> bytes:
    return c.encode("ascii")


def _batch_dims(X):
    """(batch, ncols, ld, stride) of a (batch, ncols, ld) tensor with unit inner stride."""
    if X.dim() != 3:
        raise ValueError("expected a (batch, ncols, ld) tensor")
    if X.stride(2) != 1 or X.stride(1) != X.shape[2]:
        raise ValueError("each problem must be a contiguous column-major (ncols, ld) block")
    if X.dtype.itemsize != 8:
        raise ValueError("float64 tensors expected")
    return X.shape[0], X.shape[1], X.shape[2], X.stride(0)


def _bstride(name, b, stride, batch):
    """Batch stride of an operand: its own when it holds one matrix per problem, 0 when it holds
    one matrix shared by every problem; any other batch count is refused (nothing launched)."""
    if b == batch:
        return stride if batch > 1 else 0
    if b == 1:
        return 0
    raise ValueError(f"{name} holds {b} matrices for a batch of {batch}: expected {batch} or 1")


def _square(*Xs):
    """Common order when every tensor is an unpadded square batch, else None."""
    n = Xs[0].shape[1]
    return n if all(X.shape[1] == X.shape[2] == n for X in Xs) else None


def dgemm(transa: str, transb: str, alpha: float, A, B, beta: float, C, m=None, n=None, k=None,
          stream=None):
    """C <= alpha op(A) op(B) + beta C for every problem of a strided batch (in place on C).

    m, n, k may be omitted only when A, B and C are unpadded square batches of
    one order (the leading dimension cannot tell padding from rows otherwise).
    """
    bA, cA, ldA, sA = _batch_dims(A)
    bB, cB, ldB, sB = _batch_dims(B)
    bC, cC, ldC, sC = _batch_dims(C)
    if m is None or n is None or k is None:
        sq = _square(A, B, C)
        if sq is None:
            raise ValueError("pass m, n, k explicitly for padded or non-square operands")
        m = sq if m is None else m
        n = sq if n is None else n
        k = sq if k is None else k
    _check("bf_dgemm_strided_batched", bf_dgemm_strided_batched(
        _ch(transa), _ch(transb), m, n, k, alpha, _ptr(A), ldA, _bstride("A", bA, sA, bC), _ptr(B), ldB,
        _bstride("B", bB, sB, bC), beta, _ptr(C), ldC, sC, bC, _stream(stream)))
    return C


def dtrsm(side: str, uplo: str, transa: str, diag: str, alpha: float, A, B, m=None, n=None,
          stream=None):
    """op(A) X = alpha B (side 'L') or X op(A) = alpha B (side 'R'); X overwrites B.

    m, n may be omitted only for unpadded square batches of one order.
    """
    bA, cA, ldA, sA = _batch_dims(A)
    bB, cB, ldB, sB = _batch_dims(B)
    if m is None or n is None:
        sq = _square(A, B)
        if sq is None:
            raise ValueError("pass m, n explicitly for padded or non-square operands")
        m = sq if m is None else m
        n = sq if n is None else n
    _check("bf_dtrsm_strided_batched", bf_dtrsm_strided_batched(
        _ch(side), _ch(uplo), _ch(transa), _ch(diag), m, n, alpha, _ptr(A), ldA, _bstride("A", bA, sA, bB),
        _ptr(B), ldB, sB, bB, _stream(stream)))
    return B


def dpotrf(A, n=None, info=None, uplo: str = "L", stream=None):
    """Cholesky of every problem in place (uplo 'L': A = L L^T, 'U': A = U^T U); returns info."""
    import torch
    bA, cA, ldA, sA = _batch_dims(A)
    n = cA if n is None else n
    if info is None:
        info = torch.empty(bA, dtype=torch.int32, device=A.device)
    _check("bf_dpotrf_strided_batched", bf_dpotrf_strided_batched(
        _ch(uplo), n, _ptr(A), ldA, sA, _ptr(info), bA, _stream(stream)))
    return info


def dtrfill(A, info=None, n=None, uplo: str = "L", stream=None):
    """Zero the strict triangle opposite `uplo` of every problem, and set every problem whose
    info is nonzero to NaN (in place on A)."""
    bA, cA, ldA, sA = _batch_dims(A)
    n = cA if n is None else n
    if info is not None and info.numel() != bA:
        raise ValueError(f"info holds {info.numel()} entries for a batch of {bA}")
    _check("bf_dtrfill_strided_batched", bf_dtrfill_strided_batched(
        _ch(uplo), n, _ptr(A), ldA, sA, _ptr(info) if info is not None else None, bA, _stream(stream)))
    return A


def dpotrs(L, B, n=None, nrhs=None, uplo: str = "L", stream=None):
    """Solve A X = B with the Cholesky factor L of A (in place on B)."""
    bL, cL, ldL, sL = _batch_dims(L)
    bB, cB, ldB, sB = _batch_dims(B)
    n = cL if n is None else n
    nrhs = cB if nrhs is None else nrhs
    _check("bf_dpotrs_strided_batched", bf_dpotrs_strided_batched(
        _ch(uplo), n, nrhs, _ptr(L), ldL, _bstride("L", bL, sL, bB), _ptr(B), ldB, sB, bB, _stream(stream)))
    return B


# ---------------------------------------------------------------------------- variable-size batches
def _dims2(X):
    """(ncols, ld) of one problem: a contiguous column-major (ncols, ld) float64 tensor."""
    if X.dim() != 2 or X.stride(1) != 1 or X.stride(0) != X.shape[1] or X.dtype.itemsize != 8:
        raise ValueError("each problem must be a contiguous column-major (ncols, ld) float64 tensor")
    return X.shape[0], X.shape[1]


class _DevArrays:
    """Device copies of per-problem sizes and pointers, kept alive on the launch stream."""

    def __init__(self, dev, stream):
        self.dev, self.stream, self.keep = dev, stream, []

    def ints(self, vals):
        import torch
        t = torch.tensor([int(v) for v in vals], dtype=torch.int32, device=self.dev)
        self.keep.append(t)
        return _ptr(t)

    def ptrs(self, ts):
        import torch
        t = torch.tensor([x.data_ptr() for x in ts], dtype=torch.int64, device=self.dev)
        self.keep.append(t)
        return _ptr(t)

    def done(self):
        if self.stream is not None:
            for t in self.keep:
                t.record_stream(self.stream)


def dgemm_vbatched(transa: str, transb: str, alpha: float, As, Bs, beta: float, Cs, ms, ns, ks, stream=None):
    """C_q <= alpha op(A_q) op(B_q) + beta C_q for lists of problems of different sizes (m_q, n_q,
    k_q), each matrix a column-major (ncols, ld) tensor.  Returns dinfo (per problem: 0, or
    minus the position of an illegal argument of that problem, which was skipped)."""
    import torch
    batch = len(Cs)
    dev = Cs[0].device
    d = _DevArrays(dev, stream)
    dinfo = torch.empty(batch, dtype=torch.int32, device=dev)
    _check("bf_dgemm_vbatched", bf_dgemm_vbatched(
        _ch(transa), _ch(transb), d.ints(ms), d.ints(ns), d.ints(ks), alpha, d.ptrs(As),
        d.ints(_dims2(A)[1] for A in As), d.ptrs(Bs), d.ints(_dims2(B)[1] for B in Bs), beta, d.ptrs(Cs),
        d.ints(_dims2(C)[1] for C in Cs), batch, max(ms, default=0), max(ns, default=0), max(ks, default=0),
        _ptr(dinfo), _stream(stream)))
    d.done()
    return dinfo


def dtrsm_vbatched(side: str, uplo: str, transa: str, diag: str, alpha: float, As, Bs, ms, ns, stream=None):
    """op(A_q) X = alpha B_q (side 'L') or X op(A_q) = alpha B_q (side 'R') for lists of problems
    of different sizes; X overwrites B_q.  Returns dinfo (see dgemm_vbatched)."""
    import torch
    batch = len(Bs)
    dev = Bs[0].device
    d = _DevArrays(dev, stream)
    dinfo = torch.empty(batch, dtype=torch.int32, device=dev)
    _check("bf_dtrsm_vbatched", bf_dtrsm_vbatched(
        _ch(side), _ch(uplo), _ch(transa), _ch(diag), d.ints(ms), d.ints(ns), alpha, d.ptrs(As),
        d.ints(_dims2(A)[1] for A in As), d.ptrs(Bs), d.ints(_dims2(B)[1] for B in Bs), batch,
        max(ms, default=0), max(ns, default=0), _ptr(dinfo), _stream(stream)))
    d.done()
    return dinfo


def dpotrf_vbatched(As, ns, uplo: str = "L", stream=None):
    """Cholesky (lower) of a list of problems of different orders n_q, in place; returns info
    (LAPACK info per problem, or minus the position of an illegal argument of that problem)."""
    import torch
    batch = len(As)
    dev = As[0].device
    d = _DevArrays(dev, stream)
    info = torch.empty(batch, dtype=torch.int32, device=dev)
    _check("bf_dpotrf_vbatched", bf_dpotrf_vbatched(
        _ch(uplo), d.ints(ns), d.ptrs(As), d.ints(_dims2(A)[1] for A in As), _ptr(info), batch,
        max(ns, default=0), _stream(stream)))
    d.done()
    return info


def dpotrs_vbatched(Ls, Bs, ns, nrhss, uplo: str = "L", stream=None):
    """Solve A_q X = B_q with the Cholesky factors L_q (from dpotrf / dpotrf_vbatched, same uplo)
    for lists of problems of different orders n_q and right-hand-side counts; X overwrites B_q.
    Returns dinfo (0, or minus the position of an illegal argument of that problem)."""
    import torch
    batch = len(Bs)
    dev = Bs[0].device
    d = _DevArrays(dev, stream)
    dinfo = torch.empty(batch, dtype=torch.int32, device=dev)
    _check("bf_dpotrs_vbatched", bf_dpotrs_vbatched(
        _ch(uplo), d.ints(ns), d.ints(nrhss), d.ptrs(Ls), d.ints(_dims2(L)[1] for L in Ls), d.ptrs(Bs),
        d.ints(_dims2(B)[1] for B in Bs), batch, max(ns, default=0), max(nrhss, default=0), _ptr(dinfo),
        _stream(stream)))
    d.done()
    return dinfo


def dsyrk(uplo: str, trans: str, alpha: float, A, beta: float, C, n=None, k=None, stream=None):
    """C <= alpha op(A) op(A)^T + beta C on the uplo triangle, every problem (in place on C).

    Defaults: n = C's number of columns; k = A's number of columns for trans 'N', A's leading
    dimension for 'T' (pass k when that A is padded).
    """
    bA, cA, ldA, sA = _batch_dims(A)
    bC, cC, ldC, sC = _batch_dims(C)
    n = cC if n is None else n
    if k is None:
        k = cA if trans.upper() == "N" else ldA
    _check("bf_dsyrk_strided_batched", bf_dsyrk_strided_batched(
        _ch(uplo), _ch(trans), n, k, alpha, _ptr(A), ldA, _bstride("A", bA, sA, bC), beta, _ptr(C), ldC, sC, bC,
        _stream(stream)))
    return C


def dsyrk_dpotrf(A, C, n=None, k=None, info=None, stream=None):
    """C <= chol(C + A A^T) (lower) in one kernel, every problem; returns the info tensor."""
    import torch
    bA, cA, ldA, sA = _batch_dims(A)
    bC, cC, ldC, sC = _batch_dims(C)
    n = cC if n is None else n
    k = cA if k is None else k
    if info is None:
        info = torch.empty(bC, dtype=torch.int32, device=C.device)
    _check("bf_dsyrk_dpotrf_strided_batched", bf_dsyrk_dpotrf_strided_batched(
        n, k, _ptr(A), ldA, _bstride("A", bA, sA, bC), _ptr(C), ldC, sC, _ptr(info), bC, _stream(stream)))
    return info


def dtrmm(side: str, uplo: str, transa: str, diag: str, alpha: float, A, B, m=None, n=None, stream=None):
    """B <= alpha op(A) B (side 'L') or alpha B op(A) (side 'R'), every problem (in place on B).

    m, n may be omitted only for unpadded square batches of one order.
    """
    bA, cA, ldA, sA = _batch_dims(A)
    bB, cB, ldB, sB = _batch_dims(B)
    if m is None or n is None:
        sq = _square(A, B)
        if sq is None:
            raise ValueError("pass m, n explicitly for padded or non-square operands")
        m = sq if m is None else m
        n = sq if n is None else n
    _check("bf_dtrmm_strided_batched", bf_dtrmm_strided_batched(
        _ch(side), _ch(uplo), _ch(transa), _ch(diag), m, n, alpha, _ptr(A), ldA, _bstride("A", bA, sA, bB),
        _ptr(B), ldB, sB, bB, _stream(stream)))
    return B


def dgetrf(A, n=None, ipiv=None, info=None, stream=None, m=None):
    """LU with partial pivoting of every m x n problem in place; returns (ipiv, info).

    n defaults to A's number of columns, m to n (square).  ipiv: (batch, min(m, n)) int32,
    1-based row interchanges; info: (batch,) int32.
    """
    import torch
    bA, cA, ldA, sA = _batch_dims(A)
    n = cA if n is None else n
    m = n if m is None else m
    if ipiv is None:
        ipiv = torch.empty(bA, max(min(m, n), 1), dtype=torch.int32, device=A.device)
    if info is None:
        info = torch.empty(bA, dtype=torch.int32, device=A.device)
    _check("bf_dgetrf_strided_batched", bf_dgetrf_strided_batched(
        m, n, _ptr(A), ldA, sA, _ptr(ipiv), ipiv.shape[-1], _ptr(info), bA, _stream(stream)))
    return ipiv, info


def dgetrs(trans: str, LU, ipiv, B, n=None, nrhs=None, stream=None):
    """Solve op(A) X = B with dgetrf's factors and pivots (in place on B)."""
    bL, cL, ldL, sL = _batch_dims(LU)
    bB, cB, ldB, sB = _batch_dims(B)
    n = cL if n is None else n
    nrhs = cB if nrhs is None else nrhs
    _check("bf_dgetrs_strided_batched", bf_dgetrs_strided_batched(
        _ch(trans), n, nrhs, _ptr(LU), ldL, _bstride("LU", bL, sL, bB), _ptr(ipiv),
        _bstride("ipiv", ipiv.shape[0], ipiv.shape[-1], bB), _ptr(B), ldB, sB, bB,
        _stream(stream)))
    return B


def riccati(BAt, RSQ, QN, nx: int, nu: int, F=None, info=None, fused: bool = True, work=None, stream=None):
    """Square-root Riccati recursion (section 5) for a batch of independent problems.

    BAt (batch, N, nx, m): per stage [B^T; A^T] (m x nx, column-major); RSQ (batch, N, m, m):
    [R S; S^T Q]; QN (batch, nx, nx); m = nu + nx.  Returns (F, info) with F (batch, N+1, m, m)
    the stage factors (see bf_riccati_strided_batched).
    """
    import torch
    batch, N = BAt.shape[0], BAt.shape[1]
    m = nx + nu
    if F is None:
        F = torch.empty(batch, N + 1, m, m, dtype=torch.float64, device=BAt.device)
    if info is None:
        info = torch.empty(batch, dtype=torch.int32, device=BAt.device)
    wb = bf_riccati_workspace_bytes(nx, nu, batch)
    if work is None:
        work = torch.empty(max(wb, 1), dtype=torch.uint8, device=BAt.device)
    for t in (BAt, RSQ, QN, F):
        if not t.is_contiguous():
            raise ValueError("riccati operands must be contiguous")
    _check("bf_riccati_strided_batched", bf_riccati_strided_batched(
        N, nx, nu, _ptr(BAt), N * m * nx, _ptr(RSQ), N * m * m, _ptr(QN), nx * nx, _ptr(F), (N + 1) * m * m,
        _ptr(info), 1 if fused else 0, _ptr(work), work.numel(), batch, _stream(stream)))
    return F, info


def dsposv(A, B, X=None, n=None, nrhs=None, tol: float = 1e-12, itmax: int = 30, iter=None, info=None,
           work=None, uplo: str = "L", stream=None):
    """Mixed-precision SPD solve A X = B (binary32 factor, binary64 refinement).

    `work` (a uint8 CUDA tensor of bf_dsposv_workspace_bytes(n, batch) bytes) is allocated
    when not given.  Returns (X, iter, info) with per-problem refinement counts (-1 = binary64
    fallback).
    """
    import torch
    bA, cA, ldA, sA = _batch_dims(A)
    bB, cB, ldB, sB = _batch_dims(B)
    n = cA if n is None else n
    nrhs = cB if nrhs is None else nrhs
    if X is None:
        X = torch.empty_like(B)
    bX, cX, ldX, sX = _batch_dims(X)
    if bB != bA or bX != bA:
        raise ValueError(f"A, B and X hold {bA}, {bB} and {bX} problems: one batch count expected")
    if iter is None:
        iter = torch.empty(bA, dtype=torch.int32, device=A.device)
    if info is None:
        info = torch.empty(bA, dtype=torch.int32, device=A.device)
    wb = bf_dsposv_workspace_bytes(n, bA)
    if work is None:
        work = torch.empty(max(wb, 1), dtype=torch.uint8, device=A.device)
    _check("bf_dsposv_strided_batched", bf_dsposv_strided_batched(
        _ch(uplo), n, nrhs, _ptr(A), ldA, sA, _ptr(B), ldB, sB, _ptr(X), ldX, sX, _ptr(iter), _ptr(info),
        tol, itmax, _ptr(work), work.numel(), bA, _stream(stream)))
    return X, iter, info


class RaggedPlan:
    """One persistent, graph-captured launch that factors and solves a ragged batch in place.

    ns: host int32 orders; S, B: flat float64 device tensors; offS, offB: host int64 element
    offsets (matrix b at S[offS[b]:], ld = n_b; its right-hand sides at B[offB[b]:], ld = n_b).
    The workspace and info tensors are owned by the plan object.
    """

    def __init__(self, ns, S, offS, B, offB, nrhs, lane_max=None, threads=None, stream=None):
        import numpy as np
        import torch
        lane_max = _ragged_cfg["lane_max"] if lane_max is None else lane_max
        threads = _ragged_cfg["threads"] if threads is None else threads
        self.ns = np.ascontiguousarray(ns, dtype=np.int32)
        self.offS = np.ascontiguousarray(offS, dtype=np.int64)
        self.offB = np.ascontiguousarray(offB, dtype=np.int64)
        batch = len(self.ns)
        self.S, self.B = S, B
        self.info = torch.zeros(batch, dtype=torch.int32, device=S.device)
        wb = bf_ragged_workspace_bytes(batch)
        self.work = torch.empty(wb, dtype=torch.uint8, device=S.device)
        self._plan = ctypes.c_void_p()
        _check("bf_ragged_potrf_potrs_plan_create", bf_ragged_potrf_potrs_plan_create(
            batch, self.ns.ctypes.data_as(ctypes.c_void_p), nrhs, _ptr(S),
            self.offS.ctypes.data_as(ctypes.c_void_p), _ptr(B), self.offB.ctypes.data_as(ctypes.c_void_p),
            _ptr(self.info), _ptr(self.work), wb, lane_max, threads, _stream(stream), ctypes.byref(self._plan)))

    def launch(self, stream=None):
        _check("bf_ragged_plan_launch", bf_ragged_plan_launch(self._plan, _stream(stream)))

    def describe(self):
        out = (ctypes.c_int * 5)()
        _check("bf_ragged_plan_info", bf_ragged_plan_info(self._plan, out))
        return dict(big=out[0], items=out[1], ctas=out[2], threads=out[3], smem=out[4])

    def __del__(self):
        if getattr(self, "_plan", None) and self._plan.value:
            bf_ragged_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()


def tune_query(routine: int, code: int, m: int, n: int, k: int, batch: int):
    out = (ctypes.c_int * 5)()
    _check("bf_tune_query", bf_tune_query(routine, code, m, n, k, batch, out))
    return list(out)


def tune_set(routine: int, code: int, n_lo: int, n_hi: int, variant: int, p0=0, p1=0, p2=0, p3=0):
    _check("bf_tune_set", bf_tune_set(routine, code, n_lo, n_hi, variant, p0, p1, p2, p3))


def tune_set_batch_rule(routine: int, code: int, n_lo: int, n_hi: int, cta_max: int, team4_max: int,
                        team2_max: int):
    """Measured batch-size bounds of dpotrf's small-batch forms (one problem per CTA, teams of
    4 and of 2 lanes per problem) for orders in [n_lo, n_hi]; negative keeps the built-in."""
    _check("bf_tune_set_batch_rule",
           bf_tune_set_batch_rule(routine, code, n_lo, n_hi, cta_max, team4_max, team2_max))


def tune_clear():
    bf_tune_clear()


_RAGGED_DEFAULT = {"lane_max": 32, "threads": 128}
_ragged_cfg = dict(_RAGGED_DEFAULT)


def ragged_config():
    """The ragged plan's threshold and CTA size: tuned if a table provided them, else defaults."""
    return dict(_ragged_cfg)


def load_table(path: str) -> int:
    """Install a tuned size-switch table (written by the autotuner); returns the entry count."""
    import json
    with open(path) as f:
        doc = json.load(f)
    for e in doc["entries"]:
        p = list(e["p"]) + [0] * (4 - len(e["p"]))
        tune_set(e["routine"], e["code"], e["lo"], e["hi"], e["variant"], *p[:4])
    for r in doc.get("batch_rules", []):
        tune_set_batch_rule(r["routine"], r["code"], r["lo"], r["hi"], r["cta_max"], r["team4_max"],
                            r["team2_max"])
    if "ragged" in doc:
        _ragged_cfg.update({k: int(doc["ragged"][k]) for k in ("lane_max", "threads")})
    return len(doc["entries"])


def _autoload_table():
    """Load tuned/<this GPU's name>.json if it exists (set BFGPU_NO_TUNED=1 to skip)."""
    if os.environ.get("BFGPU_NO_TUNED"):
        return None
    try:
        import torch
        if not torch.cuda.is_available():
            return None
        name = torch.cuda.get_device_name()
    except Exception:
        return None
    safe = "".join(c if c.isalnum() else "_" for c in name)
    path = os.path.join(_HERE, "tuned", safe + ".json")
    if os.path.exists(path):
        load_table(path)
        return path
    return None


TUNED_TABLE = _autoload_table()


def reset_table():
    """Remove every override and reinstall the tuned table loaded at import (if any)."""
    tune_clear()
    if TUNED_TABLE:
        load_table(TUNED_TABLE)
