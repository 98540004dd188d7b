"""CPU oracle for the batched small-matrix FP64 BLAS/LAPACK library.

TEST INFRASTRUCTURE ONLY.  This package may be imported by the test suite,
by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``;
the GPU library (``paper_1902_08115_gb300``) never imports it, and the two
share no code.  The arithmetic lives in ``bfo.c`` (plain C, binary64, natural
loop order, compiled with ``-ffp-contract=off``); this module compiles it with
gcc, loads it with ctypes and marshals numpy arrays.

Batch convention: a batch of column-major matrices with leading dimension
``ld`` and ``ncols`` columns is a C-contiguous float64 numpy array of shape
``(batch, ncols, ld)``; element (i, j) of problem b is ``X[b, j, i]``
(section 2.1, "Notation": the BLAS stores matrices column-major).

Functions and the passage each follows:

=========================  ===================================================
``dgemm``                  section 2.1, C <= alpha op(A) op(B) + beta C
``dpotrf_l``               section 3.1 "dpotrf", unblocked Cholesky, LAPACK info
``dtrsm``                  section 3.1 "dtrsm", all side/uplo/trans/diag cases
``dpotrs_l``               forward + backward substitution with the factor
``ragged_potrf_potrs``     per-problem order n[b], factor then solve
``backward_error``         Rigal-Gaches normwise backward error, FP64 residual
``dsposv``                 binary32 factor + binary64 iterative refinement
``dpotrf_l_adjoint``       reverse mode of the unblocked Cholesky loop
``spd_solve_loss_grad``    closed-form gradient of sum(A^{-1}B .* W)
``dsyrk``                  section 3.1 "dsyrk", C <= alpha op(A) op(A)^T + beta C
``dsyrk_dpotrf_l``         dsyrk then dpotrf: chol(C + A A^T) (section 5)
``dtrmm``                  section 3.1 "dtrmm", all side/uplo/trans/diag cases
``dpotrf_u``               upper Cholesky A = U^T U (appendix routine table)
``dgetrf`` / ``dgetrs``    section 3.1 "dgetrf", LU with partial pivoting + solve
``riccati``                section 5 "Riccati recursion", square-root form
=========================  ===================================================
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfo.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libbfo.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_llp = ctypes.POINTER(ctypes.c_longlong)
_c = ctypes.c_char
_i = ctypes.c_int
_ll = ctypes.c_longlong
_d = ctypes.c_double


def build(force: bool = False) -> str:
    """Compile bfo.c into a shared library (gcc -O2 -fopenmp, no FMA contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        sig = {
            "bfo_num_threads": ([], _i),
            "bfo_set_num_threads": ([_i], None),
            "bfo_dgemm": ([_c, _c, _i, _i, _i, _d, _dp, _i, _dp, _i, _d, _dp, _i], _i),
            "bfo_dgemm_sb": ([_c, _c, _i, _i, _i, _d, _dp, _i, _ll, _dp, _i, _ll, _d, _dp, _i,
                              _ll, _i], None),
            "bfo_dpotrf_l": ([_i, _dp, _i], _i),
            "bfo_dpotrf_l_sb": ([_i, _dp, _i, _ll, _i, _ip], None),
            "bfo_dtrsm": ([_c, _c, _c, _c, _i, _i, _d, _dp, _i, _dp, _i], _i),
            "bfo_dtrsm_sb": ([_c, _c, _c, _c, _i, _i, _d, _dp, _i, _ll, _dp, _i, _ll, _i], None),
            "bfo_dpotrs_l_sb": ([_i, _i, _dp, _i, _ll, _dp, _i, _ll, _i], None),
            "bfo_ragged_potrf_potrs": ([_i, _ip, _llp, _dp, _llp, _dp, _i, _ip], None),
            "bfo_backward_error_sb": ([_i, _dp, _i, _ll, _dp, _ll, _dp, _ll, _i, _dp], None),
            "bfo_dsposv_sb": ([_i, _dp, _i, _ll, _dp, _ll, _dp, _ll, _d, _i, _i, _ip, _ip], None),
            "bfo_dpotrf_l_adjoint": ([_i, _dp, _i, _dp, _i, _dp, _i], None),
            "bfo_spd_solve_loss_grad_sb": ([_i, _i, _i, _i, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                            _dp, _dp, _dp, _ip], None),
            "bfo_dsyrk": ([_c, _c, _i, _i, _d, _dp, _i, _d, _dp, _i], _i),
            "bfo_dsyrk_sb": ([_c, _c, _i, _i, _d, _dp, _i, _ll, _d, _dp, _i, _ll, _i], None),
            "bfo_dsyrk_dpotrf_l_sb": ([_i, _i, _dp, _i, _ll, _dp, _i, _ll, _i, _ip], None),
            "bfo_dtrmm": ([_c, _c, _c, _c, _i, _i, _d, _dp, _i, _dp, _i], _i),
            "bfo_dtrmm_sb": ([_c, _c, _c, _c, _i, _i, _d, _dp, _i, _ll, _dp, _i, _ll, _i], None),
            "bfo_dpotrf_u_sb": ([_i, _dp, _i, _ll, _i, _ip], None),
            "bfo_dgetrf_sb": ([_i, _i, _dp, _i, _ll, _ip, _i, _ip], None),
            "bfo_dgetrs_sb": ([_c, _i, _i, _dp, _i, _ll, _ip, _dp, _i, _ll, _i], None),
            "bfo_riccati_sb": ([_i, _i, _i, _dp, _dp, _dp, _dp, _i, _ip], None),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _f64(x: np.ndarray) -> np.ndarray:
    if x.dtype != np.float64 or not x.flags.c_contiguous:
        raise TypeError("oracle arrays must be C-contiguous float64 (batch, ncols, ld)")
    return x


def _p(x: np.ndarray):
    return x.ctypes.data_as(_dp)


def _ch(c: str) -> bytes:
    return c.encode("ascii")


def num_threads() -> int:
    return _load().bfo_num_threads()


def set_num_threads(t: int) -> None:
    _load().bfo_set_num_threads(int(t))


def _batch3(x: np.ndarray) -> np.ndarray:
    return x[None] if x.ndim == 2 else x


def dgemm(ta: str, tb: str, m: int, n: int, k: int, alpha: float, A: np.ndarray,
          B: np.ndarray, beta: float, C: np.ndarray) -> np.ndarray:
    """Batched C <= alpha op(A) op(B) + beta C (section 2.1); returns a new C."""
    A, B, C = (_f64(_batch3(x)) for x in (A, B, C))
    out = C.copy()
    batch = out.shape[0]
    lda, ldb, ldc = A.shape[2], B.shape[2], out.shape[2]
    _load().bfo_dgemm_sb(_ch(ta), _ch(tb), m, n, k, alpha, _p(A), lda, A[0].size, _p(B), ldb,
                         B[0].size, beta, _p(out), ldc, out[0].size, batch)
    return out


def dpotrf_l(A: np.ndarray, n: int | None = None):
    """Batched lower Cholesky (section 3.1 "dpotrf"); returns (factor, info)."""
    A = _f64(_batch3(A))
    out = A.copy()
    batch, ncols, lda = out.shape
    n = ncols if n is None else n
    info = np.zeros(batch, dtype=np.int32)
    _load().bfo_dpotrf_l_sb(n, _p(out), lda, out[0].size, batch, info.ctypes.data_as(_ip))
    return out, info


def dtrsm(side: str, uplo: str, ta: str, diag: str, m: int, n: int, alpha: float,
          A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Batched triangular solve (section 3.1 "dtrsm"); returns X (B is not modified)."""
    A, B = _f64(_batch3(A)), _f64(_batch3(B))
    out = B.copy()
    _load().bfo_dtrsm_sb(_ch(side), _ch(uplo), _ch(ta), _ch(diag), m, n, alpha, _p(A),
                         A.shape[2], A[0].size, _p(out), out.shape[2], out[0].size, out.shape[0])
    return out


def dpotrs_l(L: np.ndarray, B: np.ndarray, n: int, nrhs: int) -> np.ndarray:
    """Batched solve with a lower Cholesky factor: X = L^{-T} L^{-1} B."""
    L, B = _f64(_batch3(L)), _f64(_batch3(B))
    out = B.copy()
    _load().bfo_dpotrs_l_sb(n, nrhs, _p(L), L.shape[2], L[0].size, _p(out), out.shape[2],
                            out[0].size, out.shape[0])
    return out


def ragged_potrf_potrs(ns: np.ndarray, S_flat: np.ndarray, offS: np.ndarray,
                       X_flat: np.ndarray, offX: np.ndarray, nrhs: int):
    """Ragged batch: factor every S_b (order ns[b]) and solve S_b X_b = B_b in place.

    ``S_flat`` / ``X_flat`` are flat float64 arrays; problem b's matrix starts at
    ``offS[b]`` (leading dimension ns[b]) and its right-hand sides at ``offX[b]``.
    Returns (S_out, X_out, info).
    """
    ns = np.ascontiguousarray(ns, dtype=np.int32)
    offS = np.ascontiguousarray(offS, dtype=np.int64)
    offX = np.ascontiguousarray(offX, dtype=np.int64)
    S = np.array(S_flat, dtype=np.float64, copy=True)
    X = np.array(X_flat, dtype=np.float64, copy=True)
    info = np.zeros(ns.shape[0], dtype=np.int32)
    _load().bfo_ragged_potrf_potrs(ns.shape[0], ns.ctypes.data_as(_ip), offS.ctypes.data_as(_llp),
                                   _p(S), offX.ctypes.data_as(_llp), _p(X), nrhs,
                                   info.ctypes.data_as(_ip))
    return S, X, info


def backward_error(A: np.ndarray, x: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Per-problem eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    A = _f64(_batch3(A))
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(A.shape[0], -1)
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(A.shape[0], -1)
    n = A.shape[1]
    eta = np.zeros(A.shape[0], dtype=np.float64)
    _load().bfo_backward_error_sb(n, _p(A), A.shape[2], A[0].size, _p(x), x.shape[1], _p(b),
                                  b.shape[1], A.shape[0], _p(eta))
    return eta


def dsposv(A: np.ndarray, b: np.ndarray, tol: float = 1e-12, itmax: int = 30):
    """Mixed-precision SPD solve (binary32 factor, binary64 refinement), one RHS.

    Returns (x, iters, info); iters[p] = -1 marks a binary64 fallback.
    """
    A = _f64(_batch3(A))
    batch, n, lda = A.shape
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(batch, -1)
    x = np.zeros((batch, n), dtype=np.float64)
    iters = np.zeros(batch, dtype=np.int32)
    info = np.zeros(batch, dtype=np.int32)
    _load().bfo_dsposv_sb(n, _p(A), lda, A[0].size, _p(b), b.shape[1], _p(x), n, tol, itmax,
                          batch, iters.ctypes.data_as(_ip), info.ctypes.data_as(_ip))
    return x, iters, info


def dpotrf_l_adjoint(L: np.ndarray, Lbar: np.ndarray) -> np.ndarray:
    """Reverse mode of the unblocked Cholesky: lower-triangular d(loss)/dA (one problem)."""
    L = np.ascontiguousarray(L, dtype=np.float64)
    Lbar = np.ascontiguousarray(Lbar, dtype=np.float64)
    ncols, ld = L.shape
    Abar = np.zeros((ncols, ncols), dtype=np.float64)
    _load().bfo_dpotrf_l_adjoint(ncols, _p(L), ld, _p(Lbar), Lbar.shape[1], _p(Abar), ncols)
    return Abar


def spd_solve_loss_grad(Qd: np.ndarray, J: np.ndarray, B: np.ndarray, W: np.ndarray):
    """Closed-form gradient of loss = sum((Q + J J^T)^{-1} B .* W), batched.

    Shapes (column-major per problem): Qd (batch, n), J (batch, q, n),
    B and W (batch, r, n).  Returns a dict with X, loss, Jbar, Qbar, Bbar, Wbar, info.
    """
    Qd = np.ascontiguousarray(Qd, dtype=np.float64)
    J, B, W = (_f64(x) for x in (J, B, W))
    batch, n = Qd.shape
    q, r = J.shape[1], B.shape[1]
    X = np.zeros_like(B)
    loss = np.zeros(batch)
    Jbar = np.zeros_like(J)
    Qbar = np.zeros_like(Qd)
    Bbar = np.zeros_like(B)
    Wbar = np.zeros_like(W)
    info = np.zeros(batch, dtype=np.int32)
    _load().bfo_spd_solve_loss_grad_sb(n, q, r, batch, _p(Qd), _p(J), _p(B), _p(W), _p(X),
                                       _p(loss), _p(Jbar), _p(Qbar), _p(Bbar), _p(Wbar),
                                       info.ctypes.data_as(_ip))
    return dict(X=X, loss=loss, Jbar=Jbar, Qbar=Qbar, Bbar=Bbar, Wbar=Wbar, info=info)


def dsyrk(uplo: str, trans: str, n: int, k: int, alpha: float, A: np.ndarray, beta: float,
          C: np.ndarray) -> np.ndarray:
    """Batched C <= alpha op(A) op(A)^T + beta C on the uplo triangle (section 3.1 "dsyrk")."""
    A, C = _f64(_batch3(A)), _f64(_batch3(C))
    out = C.copy()
    _load().bfo_dsyrk_sb(_ch(uplo), _ch(trans), n, k, alpha, _p(A), A.shape[2], A[0].size, beta,
                         _p(out), out.shape[2], out[0].size, out.shape[0])
    return out


def dsyrk_dpotrf_l(n: int, k: int, A: np.ndarray, C: np.ndarray):
    """Batched chol(C + A A^T), lower (dsyrk_ln then dpotrf_l); returns (factor, info)."""
    A, C = _f64(_batch3(A)), _f64(_batch3(C))
    out = C.copy()
    info = np.zeros(out.shape[0], dtype=np.int32)
    _load().bfo_dsyrk_dpotrf_l_sb(n, k, _p(A), A.shape[2], A[0].size, _p(out), out.shape[2], out[0].size,
                                  out.shape[0], info.ctypes.data_as(_ip))
    return out, info


def dtrmm(side: str, uplo: str, ta: str, diag: str, m: int, n: int, alpha: float, A: np.ndarray,
          B: np.ndarray) -> np.ndarray:
    """Batched triangular multiply (section 3.1 "dtrmm"); returns the new B."""
    A, B = _f64(_batch3(A)), _f64(_batch3(B))
    out = B.copy()
    _load().bfo_dtrmm_sb(_ch(side), _ch(uplo), _ch(ta), _ch(diag), m, n, alpha, _p(A), A.shape[2],
                         A[0].size, _p(out), out.shape[2], out[0].size, out.shape[0])
    return out


def dpotrf_u(A: np.ndarray, n: int | None = None):
    """Batched upper Cholesky A = U^T U; returns (factor, info)."""
    A = _f64(_batch3(A))
    out = A.copy()
    batch, ncols, lda = out.shape
    n = ncols if n is None else n
    info = np.zeros(batch, dtype=np.int32)
    _load().bfo_dpotrf_u_sb(n, _p(out), lda, out[0].size, batch, info.ctypes.data_as(_ip))
    return out, info


def dgetrf(A: np.ndarray, m: int | None = None, n: int | None = None):
    """Batched LU with partial pivoting (section 3.1 "dgetrf"); returns (LU, ipiv, info).

    ipiv is (batch, min(m, n)) int32, 1-based as in LAPACK.
    """
    A = _f64(_batch3(A))
    out = A.copy()
    batch, ncols, lda = out.shape
    m = lda if m is None else m
    n = ncols if n is None else n
    ipiv = np.zeros((batch, min(m, n)), dtype=np.int32)
    info = np.zeros(batch, dtype=np.int32)
    _load().bfo_dgetrf_sb(m, n, _p(out), lda, out[0].size, ipiv.ctypes.data_as(_ip), batch,
                          info.ctypes.data_as(_ip))
    return out, ipiv, info


def dgetrs(trans: str, LU: np.ndarray, ipiv: np.ndarray, B: np.ndarray, n: int, nrhs: int) -> np.ndarray:
    """Batched solve op(A) X = B with dgetrf's factors; returns X."""
    LU, B = _f64(_batch3(LU)), _f64(_batch3(B))
    ipiv = np.ascontiguousarray(ipiv, dtype=np.int32).reshape(LU.shape[0], -1)
    out = B.copy()
    _load().bfo_dgetrs_sb(_ch(trans), n, nrhs, _p(LU), LU.shape[2], LU[0].size, ipiv.ctypes.data_as(_ip),
                          _p(out), out.shape[2], out[0].size, out.shape[0])
    return out


def riccati(BAt: np.ndarray, RSQ: np.ndarray, QN: np.ndarray, nx: int, nu: int):
    """Square-root Riccati recursion (section 5), batched.

    BAt (batch, N, nx, nu+nx): [B^T; A^T] per stage, column-major (nx columns);
    RSQ (batch, N, nu+nx, nu+nx): [R S; S^T Q] per stage; QN (batch, nx, nx).
    Returns (F, info): F (batch, N+1, nu+nx, nu+nx) holds every stage's Cholesky factor
    (lower triangle; stage N: chol(Q_N) in its top-left nx x nx block).
    """
    BAt = np.ascontiguousarray(BAt, dtype=np.float64)
    RSQ = np.ascontiguousarray(RSQ, dtype=np.float64)
    QN = np.ascontiguousarray(QN, dtype=np.float64)
    batch, N = BAt.shape[0], BAt.shape[1]
    m = nx + nu
    F = np.zeros((batch, N + 1, m, m), dtype=np.float64)
    info = np.zeros(batch, dtype=np.int32)
    _load().bfo_riccati_sb(N, nx, nu, _p(BAt), _p(RSQ), _p(QN), _p(F), batch, info.ctypes.data_as(_ip))
    return F, info
