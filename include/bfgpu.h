/*
 * bfgpu.h -- C ABI of the batched small-matrix FP64 BLAS/LAPACK library for
 * one GB300 (sm_103a).
 *
 * The routines keep the BLAS/LAPACK calling conventions that the paper keeps
 * for its "BLAS API" (section 1; section 2.1 "Notation"): column-major
 * storage with a leading dimension, char options ('N'/'T', 'L'/'U', ...),
 * destructive in-place output.  Every call additionally exists in batched
 * forms.  Each call switches by size between kernel variants (section 2.4,
 * "Proposed approach"): a direct kernel on the column-major operands, and
 * kernels that first pack operands into a panel layout in shared memory.
 *
 * Conventions shared by every entry point:
 *  - Pointers to matrices, pointer arrays and info arrays are DEVICE
 *    pointers owned by the caller; the library never allocates device memory
 *    on the call path (the paper's variants avoid dynamic allocation for
 *    small sizes, section 2.2 algorithm 'C').
 *  - Element (i, j) of a matrix X with leading dimension ldx is X[i + j*ldx].
 *  - Strided batches: problem b's matrix starts at X + b*strideX.
 *    Pointer-array batches: problem b's matrix starts at Xarray[b].
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL is the
 *    legacy default stream).
 *  - Return value: 0 on success; -i when the i-th argument (1-based position
 *    in the call's argument list) is illegal, in which case nothing is
 *    launched (LAPACK's info < 0 rule); BF_ERR_CUDA when a launch failed;
 *    BF_ERR_NOT_SUPPORTED for a legal option this library does not implement.
 *  - Numerical failures are reported per problem in a device `info` array
 *    (LAPACK's info > 0 rule); calls never abort or trap.
 */
#ifndef BFGPU_H
#define BFGPU_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* bf_stream_t; /* identical to cudaStream_t */

#define BF_SUCCESS 0
#define BF_ERR_CUDA 1001
#define BF_ERR_NOT_SUPPORTED 1002
#define BF_ERR_NOALLOC_LIMIT 1003

#define BF_ROUTINE_DGEMM 0
#define BF_ROUTINE_DTRSM 1
#define BF_ROUTINE_DPOTRF 2
#define BF_ROUTINE_DGETRF 3  /* code 0; variants DIRECT (lane LU) and CTA */

/* Kernel variants of the size switch (values of `variant` in bf_tune_set). */
#define BF_VARIANT_DIRECT 0  /* native column-major operands, no packing (algorithm 'D') */
#define BF_VARIANT_PACKED 1  /* operands packed into shared-memory panels ('B'/'C')     */
#define BF_VARIANT_BLOCKED 2 /* dpotrf only: right-looking sequence of the above kernels */
#define BF_VARIANT_TINY 3    /* dgemm (m, n, k <= 4) and dtrsm (orders <= 8): one thread   */
                             /* per problem, problems staged through shared memory       */
#define BF_VARIANT_CTA 4     /* one problem per CTA, for batches too small to fill the GPU */
                             /* one problem per thread: dpotrf 'L' (n <= 256, left-looking */
                             /* by 16-column panels), dgetrf (n <= 1024, right-looking by  */
                             /* 16-column panels)                                         */
#define BF_VARIANT_TEAM 5    /* dpotrf: 2 or 4 lanes of a warp per problem (p2), for      */
                             /* batches between the CTA form's and the lane form's ranges; */
                             /* dgetrf (n <= 16): 4 lanes per problem, 8 problems of a    */
                             /* warp in shared memory                                     */
#define BF_VARIANT_GROUP 6   /* dpotrf only: a group of problems per CTA in shared memory, */
                             /* the unblocked recurrence element-parallel over the group  */
                             /* (small batches of small orders)                           */
#define BF_TUNE_FORCE 0x100  /* or'ed into `variant`: the entry holds at every batch size; */
                             /* without it, dpotrf batches too small to fill the GPU one  */
                             /* problem per thread still switch to BF_VARIANT_CTA, to     */
                             /* BF_VARIANT_TEAM (12 <= n <= 64) or to BF_VARIANT_BLOCKED  */
                             /* (n > 64, batch < 20000)                                   */

/* ------------------------------------------------------------------------ */
/* dgemm (section 2.1): C <= alpha * op(A) * op(B) + beta * C,               */
/* op(X) = X ('N') or X^T ('T'); C is m x n, op(A) m x k, op(B) k x n.        */
/* beta == 0: C is written without being read.  alpha == 0 or k == 0: C is   */
/* only scaled by beta.  lda >= max(1, rows of A), ldb >= max(1, rows of B), */
/* ldc >= max(1, m).                                                         */
/* ------------------------------------------------------------------------ */
int bf_dgemm(char transa, char transb, int m, int n, int k, double alpha,
             const double* A, int lda, const double* B, int ldb, double beta,
             double* C, int ldc, bf_stream_t stream);

/* strideC >= ldc*n when batch > 1 (outputs may not overlap); strideA and    */
/* strideB may be 0 (the same operand for every problem).                    */
int bf_dgemm_strided_batched(char transa, char transb, int m, int n, int k, double alpha,
                             const double* A, int lda, long long strideA,
                             const double* B, int ldb, long long strideB, double beta,
                             double* C, int ldc, long long strideC, int batch,
                             bf_stream_t stream);

/* Aarray, Barray, Carray: device arrays of `batch` device pointers. */
int bf_dgemm_batched(char transa, char transb, int m, int n, int k, double alpha,
                     const double* const* Aarray, int lda, const double* const* Barray, int ldb,
                     double beta, double* const* Carray, int ldc, int batch, bf_stream_t stream);

/* Variable-size batches ("vbatched"; the paper's sizes are known only at run time, section */
/* 1).  Problem q has its own sizes m[q], n[q], k[q], leading dimensions lda[q], ldb[q],     */
/* ldc[q] and matrices Aarray[q], Barray[q], Carray[q]: all device arrays of `batch`        */
/* entries.  max_m, max_n, max_k bound the sizes over the batch (they size the launch).     */
/* A problem whose own arguments are illegal (a size < 0 or above its bound, a leading     */
/* dimension too small, a null matrix that would be read or written) is skipped and         */
/* dinfo[q] = minus that argument's position in this call (-3 m, -4 n, -5 k, -7 A, -8 lda,  */
/* -9 B, -10 ldb, -12 C, -13 ldc); else dinfo[q] = 0.  dinfo (device) may be NULL.  The     */
/* return value reports the call's own arguments (transa, transb, batch, max_*, and the     */
/* device arrays themselves being non-null when batch > 0) as the uniform calls do.         */
int bf_dgemm_vbatched(char transa, char transb, const int* m, const int* n, const int* k, double alpha,
                      const double* const* Aarray, const int* lda, const double* const* Barray,
                      const int* ldb, double beta, double* const* Carray, const int* ldc, int batch,
                      int max_m, int max_n, int max_k, int* dinfo, bf_stream_t stream);

/* ------------------------------------------------------------------------ */
/* dtrsm (section 3.1 "dtrsm"): solve op(A) X = alpha B (side 'L') or         */
/* X op(A) = alpha B (side 'R'); X overwrites B (m x n).  A is triangular    */
/* ('L' lower / 'U' upper stored), diag 'U' = unit diagonal (not read).       */
/* A is m x m for side 'L' and n x n for side 'R'; lda >= max(1, that order),*/
/* ldb >= max(1, m).  alpha == 0 sets B to zero without reading A.           */
/* ------------------------------------------------------------------------ */
int bf_dtrsm(char side, char uplo, char transa, char diag, int m, int n, double alpha,
             const double* A, int lda, double* B, int ldb, bf_stream_t stream);

int bf_dtrsm_strided_batched(char side, char uplo, char transa, char diag, int m, int n,
                             double alpha, const double* A, int lda, long long strideA,
                             double* B, int ldb, long long strideB, int batch,
                             bf_stream_t stream);

int bf_dtrsm_batched(char side, char uplo, char transa, char diag, int m, int n, double alpha,
                     const double* const* Aarray, int lda, double* const* Barray, int ldb,
                     int batch, bf_stream_t stream);

/* Variable-size dtrsm (see bf_dgemm_vbatched): per problem m[q], n[q], lda[q], ldb[q],    */
/* Aarray[q], Barray[q]; dinfo[q] = 0 or -5 m, -6 n, -8 A, -9 lda, -10 B, -11 ldb.          */
int bf_dtrsm_vbatched(char side, char uplo, char transa, char diag, const int* m, const int* n,
                      double alpha, const double* const* Aarray, const int* lda, double* const* Barray,
                      const int* ldb, int batch, int max_m, int max_n, int* dinfo, bf_stream_t stream);

/* ------------------------------------------------------------------------ */
/* dpotrf (section 3.1 "dpotrf"): Cholesky factorisation A = L L^T of SPD    */
/* matrices, uplo 'L': the lower triangle of A is read and overwritten by L; */
/* the strict upper triangle and the padding rows (lda > n) are not touched. */
/* info (device, one int per problem): 0 on success, j > 0 when the leading  */
/* minor of order j is not positive definite (or NaN); that problem's        */
/* factorisation stops at column j.  info may be NULL.  uplo 'U' (the        */
/* appendix's dpotrf_u, chol(Q, 'upper')): A = U^T U from the upper triangle, */
/* which U overwrites; the strict lower triangle is not touched.             */
/* ------------------------------------------------------------------------ */
int bf_dpotrf(char uplo, int n, double* A, int lda, int* info, bf_stream_t stream);

int bf_dpotrf_strided_batched(char uplo, int n, double* A, int lda, long long strideA,
                              int* info, int batch, bf_stream_t stream);

int bf_dpotrf_batched(char uplo, int n, double* const* Aarray, int lda, int* info, int batch,
                      bf_stream_t stream);

/* Variable-size dpotrf (see bf_dgemm_vbatched): per problem n[q], lda[q], Aarray[q];      */
/* uplo 'L' (A = L L^T) or 'U' (A = U^T U), as bf_dpotrf.  info[q] = the LAPACK info (>= 0),*/
/* or -2 (n[q] < 0 or above max_n) / -4 (lda[q] too small) for a skipped problem.  max_n    */
/* above BF_VBATCHED_POTRF_NMAX returns BF_ERR_NOT_SUPPORTED (nothing launched).           */
#define BF_VBATCHED_POTRF_NMAX 1024
int bf_dpotrf_vbatched(char uplo, const int* n, double* const* Aarray, const int* lda, int* info, int batch,
                       int max_n, bf_stream_t stream);

/* ------------------------------------------------------------------------ */
/* dsyrk (section 3.1 "dsyrk": dgemm whose A and B coincide):               */
/*   C <= alpha op(A) op(A)^T + beta C   on the uplo triangle of C           */
/* C n x n (ldc >= max(1, n)); op(A) = A (n x k, lda >= max(1, n)) for trans */
/* 'N', A^T (A stored k x n, lda >= max(1, k)) for 'T'.  The other triangle  */
/* of C is not written.  beta == 0: C is not read; alpha == 0 or k == 0:     */
/* C <= beta C on the triangle (A not read).                                 */
/* ------------------------------------------------------------------------ */
int bf_dsyrk(char uplo, char trans, int n, int k, double alpha, const double* A, int lda, double beta,
             double* C, int ldc, bf_stream_t stream);

int bf_dsyrk_strided_batched(char uplo, char trans, int n, int k, double alpha, const double* A, int lda,
                             long long strideA, double beta, double* C, int ldc, long long strideC,
                             int batch, bf_stream_t stream);

int bf_dsyrk_batched(char uplo, char trans, int n, int k, double alpha, const double* const* Aarray,
                     int lda, double beta, double* const* Carray, int ldc, int batch, bf_stream_t stream);

/* ------------------------------------------------------------------------ */
/* dsyrk + dpotrf, lower, fused (the routine of the paper's own API that     */
/* section 5 credits in the Riccati recursion): C <= chol(C + A A^T), A n x k */
/* (lda >= max(1, n)), C n x n with its lower triangle read and overwritten  */
/* by the factor (ldc >= max(1, n)); A A^T is added inside the Cholesky's    */
/* own register tiles and never stored.  info (device, may be NULL) as       */
/* bf_dpotrf.                                                                */
/* ------------------------------------------------------------------------ */
int bf_dsyrk_dpotrf(int n, int k, const double* A, int lda, double* C, int ldc, int* info,
                    bf_stream_t stream);

int bf_dsyrk_dpotrf_strided_batched(int n, int k, const double* A, int lda, long long strideA, double* C,
                                    int ldc, long long strideC, int* info, int batch, bf_stream_t stream);

/* ------------------------------------------------------------------------ */
/* dtrmm (section 3.1 "dtrmm", built like dtrsm): B <= alpha op(A) B (side   */
/* 'L', A m x m) or B <= alpha B op(A) (side 'R', A n x n); B m x n, ldb >=  */
/* max(1, m).  uplo: the stored triangle of A; diag 'U': unit diagonal, not  */
/* read.  alpha == 0: B <= 0 (A not read).                                   */
/* ------------------------------------------------------------------------ */
int bf_dtrmm(char side, char uplo, char transa, char diag, int m, int n, double alpha, const double* A,
             int lda, double* B, int ldb, bf_stream_t stream);

int bf_dtrmm_strided_batched(char side, char uplo, char transa, char diag, int m, int n, double alpha,
                             const double* A, int lda, long long strideA, double* B, int ldb,
                             long long strideB, int batch, bf_stream_t stream);

int bf_dtrmm_batched(char side, char uplo, char transa, char diag, int m, int n, double alpha,
                     const double* const* Aarray, int lda, double* const* Barray, int ldb, int batch,
                     bf_stream_t stream);

/* ------------------------------------------------------------------------ */
/* dgetrf (section 3.1 "dgetrf"): LU factorisation with partial (row)        */
/* pivoting, P A = L U, of m x n matrices.  L (m x min(m, n), unit lower     */
/* trapezoidal, below the diagonal) and U (min(m, n) x n, upper trapezoidal) */
/* overwrite A.  m != n needs m <= 1024 (else BF_ERR_NOT_SUPPORTED).         */
/* ipiv (device, min(m, n) ints per problem, stride strideIpiv >= min(m, n)):*/
/* row j was interchanged with row ipiv[j] - 1 (1-based, as LAPACK); the     */
/* pivot is the first row of largest magnitude.  info (device, may be        */
/* NULL): 0, or j when U(j-1, j-1) is exactly zero (the factorisation still   */
/* completes).                                                               */
/* ------------------------------------------------------------------------ */
int bf_dgetrf(int m, int n, double* A, int lda, int* ipiv, int* info, bf_stream_t stream);

int bf_dgetrf_strided_batched(int m, int n, double* A, int lda, long long strideA, int* ipiv,
                              long long strideIpiv, int* info, int batch, bf_stream_t stream);

/* ------------------------------------------------------------------------ */
/* dgetrs: solve op(A) X = B with the factors and pivots of bf_dgetrf:       */
/* 'N': the interchanges, L Y = P B, U X = Y;  'T': U^T Y = B, L^T Z = Y,    */
/* then the interchanges in reverse.  B (n x nrhs, ldb >= max(1, n)) is      */
/* overwritten by X.                                                         */
/* ------------------------------------------------------------------------ */
int bf_dgetrs(char trans, int n, int nrhs, const double* A, int lda, const int* ipiv, double* B, int ldb,
              bf_stream_t stream);

int bf_dgetrs_strided_batched(char trans, int n, int nrhs, const double* A, int lda, long long strideA,
                              const int* ipiv, long long strideIpiv, double* B, int ldb, long long strideB,
                              int batch, bf_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Riccati recursion, square-root form (section 5 "Riccati recursion"), for   */
/* a batch of independent problems of N stages, nx states, nu controls,      */
/* m = nu + nx.  Per problem (column-major, all leading dimensions m except  */
/* Q_N's, nx):                                                               */
/*   BAt   stage s at BAt + s m nx: [B_s^T; A_s^T], m x nx                    */
/*   RSQ   stage s at RSQ + s m m:  [R_s S_s; S_s^T Q_s], m x m, lower read   */
/*   QN    nx x nx, lower read                                              */
/*   F     stage s at F + s m m, s = 0..N: receives chol(RSQ_s + C_s C_s^T)   */
/*         with C_s = [B_s^T; A_s^T] Lc_{s+1} (dtrmm_rlnn), Lc_s its trailing */
/*         nx x nx block; F_N holds chol(Q_N) in its top-left block, zeros    */
/*         elsewhere.  Only lower triangles of F are meaningful.             */
/*   info  (device) 0, or 1000 s + j for the first stage s (N: the terminal  */
/*         factorisation) whose dpotrf failed at column j                    */
/*   fused 1: the fused dsyrk + dpotrf; 0: dsyrk then dpotrf (BLAS/LAPACK)   */
/*   work  caller-owned device memory of bf_riccati_workspace_bytes(nx, nu,  */
/*         batch) bytes                                                      */
/* The stages run as a sequence of batched launches on `stream`.            */
/* ------------------------------------------------------------------------ */
size_t bf_riccati_workspace_bytes(int nx, int nu, int batch);

int bf_riccati_strided_batched(int N, int nx, int nu, const double* BAt, long long strideBAt,
                               const double* RSQ, long long strideRSQ, const double* QN,
                               long long strideQN, double* F, long long strideF, int* info, int fused,
                               void* work, size_t work_bytes, int batch, bf_stream_t stream);

/* ------------------------------------------------------------------------ */
/* dpotrs: solve A X = B with the factor from bf_dpotrf: 'L' the forward    */
/* solve L Y = B then the backward solve L^T X = Y, 'U' U^T Y = B then       */
/* U X = Y (section 3.1 "dtrsm" left variants).  B (n x nrhs, ldb >=         */
/* max(1, n)) is overwritten by X.                                           */
/* ------------------------------------------------------------------------ */
int bf_dpotrs(char uplo, int n, int nrhs, const double* A, int lda, double* B, int ldb,
              bf_stream_t stream);

int bf_dpotrs_batched(char uplo, int n, int nrhs, const double* const* Aarray, int lda,
                      double* const* Barray, int ldb, int batch, bf_stream_t stream);
/* Variable-size dpotrs (see bf_dgemm_vbatched): per problem n[q], nrhs[q], lda[q], ldb[q],  */
/* Aarray[q] (the factor from bf_dpotrf or bf_dpotrf_vbatched with the same uplo),         */
/* Barray[q] (n[q] x nrhs[q], overwritten by X); max_n, max_nrhs bound the sizes.  dinfo[q] */
/* = 0, or -2 n, -3 nrhs, -4 A, -5 lda, -6 B, -7 ldb for a skipped problem.               */
int bf_dpotrs_vbatched(char uplo, const int* n, const int* nrhs, const double* const* Aarray,
                       const int* lda, double* const* Barray, const int* ldb, int batch, int max_n,
                       int max_nrhs, int* dinfo, bf_stream_t stream);
int bf_dpotrs_strided_batched(char uplo, int n, int nrhs, const double* A, int lda,
                              long long strideA, double* B, int ldb, long long strideB,
                              int batch, bf_stream_t stream);

/* ------------------------------------------------------------------------ */
/* dsposv (LAPACK's name for the mixed-precision SPD solve; the routines it */
/* runs are the paper's dpotrf and dtrsm, section 3.1, in binary32): solve   */
/* A X = B for SPD A (uplo 'L': lower triangle referenced, A not modified).  */
/* A is rounded to binary32 (to nearest, subnormals kept) and factored in    */
/* binary32, one problem per CTA; each pivot's square root is the correctly  */
/* rounded binary32 root, which equals the binary64 root rounded to binary32.*/
/* The binary32 solution is refined                                         */
/* in binary64 (residual b - A x and update x + d in binary64) until the     */
/* normwise backward error ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)*/
/* <= tol for every column, at most itmax steps.  If the binary32           */
/* factorisation fails (non-positive or NaN pivot, or an entry beyond the    */
/* binary32 range) or the refinement does not converge, that problem is      */
/* solved in binary64 instead.                                               */
/*   work: device memory of at least bf_dsposv_workspace_bytes(n, batch)     */
/*         bytes, 256-byte aligned, owned by the caller (LAPACK's swork: the */
/*         binary32 factors); its contents are undefined on return.          */
/*   iter[b] (device, may be NULL): refinement steps taken (max over         */
/*         columns; 0 = the binary32 solution met tol), -1 = binary64        */
/*         fallback.  info[b] (device, may be NULL): 0, or j > 0 when the    */
/*         binary64 fallback found the leading minor of order j not positive */
/*         definite (X is then not written).                                 */
/* 1 <= n <= BF_DSPOSV_NMAX (larger n: BF_ERR_NOT_SUPPORTED); ldb, ldx >= n. */
/* ------------------------------------------------------------------------ */
#define BF_DSPOSV_NMAX 256

size_t bf_dsposv_workspace_bytes(int n, int batch);
int bf_dsposv_strided_batched(char uplo, int n, int nrhs, const double* A, int lda,
                              long long strideA, const double* B, int ldb, long long strideB,
                              double* X, int ldx, long long strideX, int* iter, int* info,
                              double tol, int itmax, void* work, size_t work_bytes, int batch,
                              bf_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Reverse mode (adjoints) of the routines above, strided batches.  Output   */
/* arrays are overwritten; NULL outputs are skipped.                         */
/*                                                                           */
/* dgemm, C = alpha op(A) op(B) + beta C0 (section 2.1): given Cbar,          */
/*   Abar = alpha Cbar op(B)^T (its transpose when transa = 'T'),            */
/*   Bbar = alpha op(A)^T Cbar (its transpose when transb = 'T'),            */
/*   C0bar = beta Cbar.  Abar/Bbar have the shapes (and leading dims) of A/B. */
/* ------------------------------------------------------------------------ */
int bf_dgemm_backward_strided_batched(char transa, char transb, int m, int n, int k, double alpha,
                                      const double* A, int lda, long long strideA,
                                      const double* B, int ldb, long long strideB, double beta,
                                      const double* Cbar, int ldcb, long long strideCbar,
                                      double* Abar, int ldab, long long strideAbar,
                                      double* Bbar, int ldbb, long long strideBbar,
                                      double* C0bar, int ldc0b, long long strideC0bar, int batch,
                                      bf_stream_t stream);

/* dtrsm (section 3.1 "dtrsm"), op(A) X = alpha B or X op(A) = alpha B with   */
/* the solution X: on entry XBbar holds Xbar, on exit Bbar = alpha Z, where  */
/* op(A)^T Z = Xbar (side 'L') or Z op(A)^T = Xbar (side 'R').  Abar (may be  */
/* NULL) receives -Z X^T (side 'L') or -X^T Z (side 'R'), transposed when     */
/* transa = 'T', on the stored triangle of A only (without the diagonal when */
/* diag = 'U'); its other triangle is not written.  alpha == 0: -7.          */
int bf_dtrsm_backward_strided_batched(char side, char uplo, char transa, char diag, int m, int n,
                                      double alpha, const double* A, int lda, long long strideA,
                                      const double* X, int ldx, long long strideX,
                                      double* XBbar, int ldxb, long long strideXB,
                                      double* Abar, int ldab, long long strideAbar, int batch,
                                      bf_stream_t stream);

/* dpotrf (section 3.1 "dpotrf"), A = L L^T: given L (lower triangle read)   */
/* and Lbar (lower triangle read), writes the symmetric gradient             */
/* Abar = (S + S^T)/2, S = L^{-T} Phi(L^T Lbar) L^{-1}, Phi = lower triangle */
/* with halved diagonal (I. Murray, "Differentiation of the Cholesky         */
/* decomposition", 2016), to the full n x n of Abar (Abar must not alias L  */
/* or Lbar).  Orders up to 32 run it as one kernel, one warp per problem.   */
/* uplo 'U' (A = U^T U): L and Lbar hold U and Ubar in their upper triangles */
/* (read as L = U^T, Lbar = Ubar^T); the gradient is the same symmetric one. */
int bf_dpotrf_backward_strided_batched(char uplo, int n, const double* L, int ldl, long long strideL,
                                       const double* Lbar, int ldlb, long long strideLbar,
                                       double* Abar, int ldab, long long strideAbar, int batch,
                                       bf_stream_t stream);

/* dpotrs (section 3.1 "dtrsm", the two solves after dpotrf), A = L L^T:     */
/* X = L^{-T} Y with Y = L^{-1} B ('U', A = U^T U: X = U^{-1} Y, Y = U^{-T} B);*/
/* given the factor L, the solution X and the intermediate Y (n x nrhs each, */
/* as the forward solves left them), and Xbar in XBbar on entry:             */
/*   Z1 solves L Z1 = Xbar (the gradient of Y), Z2 solves L^T Z2 = Z1;        */
/*   on exit XBbar holds Bbar = Z2, and Lbar (n x n, must not alias the      */
/*   other arrays) receives the two solves' triangle gradients summed,       */
/*   -(X Z1^T + Z2 Y^T) on the lower triangle ('U': -(Z1 X^T + Y Z2^T) on    */
/*   the upper one), with zeros in the other strict triangle, so that all    */
/*   n x n of Lbar are written.  This equals the sum of the Abar outputs of  */
/*   the two bf_dtrsm_backward_strided_batched calls of those solves, in one */
/*   buffer and without the separate sum.  Errors: the argument's -position  */
/*   (LAPACK convention), BF_ERR_CUDA on a launch failure.                   */
int bf_dpotrs_backward_strided_batched(char uplo, int n, int nrhs, const double* L, int ldl,
                                       long long strideL, const double* X, int ldx, long long strideX,
                                       const double* Y, int ldy, long long strideY,
                                       double* XBbar, int ldxb, long long strideXB,
                                       double* Lbar, int ldlb, long long strideLbar, int batch,
                                       bf_stream_t stream);

/* After dpotrf (section 3.1 "dpotrf"; LAPACK leaves the other triangle     */
/* untouched and a failed problem's later columns unspecified), make each    */
/* problem of A a clean triangular factor: the strict triangle opposite uplo */
/* ('L': the strict upper one) is set to zero, and a problem whose info[q]  */
/* is nonzero (info: device array of batch ints, may be NULL) has its whole  */
/* n x n set to NaN, so a failed factorisation cannot be used as a finite    */
/* factor (e.g. by a gradient).  Padding rows are not touched.               */
int bf_dtrfill_strided_batched(char uplo, int n, double* A, int lda, long long strideA,
                               const int* info, int batch, bf_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Ragged batches (problems of different orders; no counterpart in the       */
/* paper, which treats one matrix per call): factor every SPD matrix with     */
/* dpotrf ('L') and solve S_b X_b = B_b (nrhs columns) in place, in ONE       */
/* persistent kernel launch captured in a CUDA graph.                        */
/*   n_host[b]      order of problem b (host array, read at plan creation)   */
/*   S + offS_host[b]  its matrix, column-major with leading dimension n_b   */
/*   B + offB_host[b]  its n_b x nrhs right-hand sides (ld n_b), overwritten  */
/*   info[b]        (device) LAPACK info of problem b                        */
/*   workspace      device memory of bf_ragged_workspace_bytes(batch) bytes, */
/*                  owned by the caller, kept for the plan's lifetime        */
/*   lane_max       orders <= lane_max are factored one problem per thread,  */
/*                  larger ones (at most 256) one problem per CTA            */
/*   threads        CTA size: 64, 128, 256 or 512                            */
/* Plan creation sorts the problems (largest first), copies the queue into   */
/* the workspace on `stream` (synchronously) and instantiates the graph; the */
/* device pointers and offsets are fixed in the plan.  bf_ragged_plan_launch */
/* enqueues the graph on `stream`.  A batch with an order above both        */
/* lane_max and 256 returns BF_ERR_NOT_SUPPORTED (nothing is launched).      */
/* bf_ragged_plan_info writes {BIG problems,                                 */
/* queue items, CTAs, threads, shared bytes} into out[5].                    */
/* ------------------------------------------------------------------------ */
typedef struct bf_ragged_plan_st* bf_ragged_plan_t;

size_t bf_ragged_workspace_bytes(int batch);
int bf_ragged_potrf_potrs_plan_create(int batch, const int* n_host, int nrhs, double* S,
                                      const long long* offS_host, double* B,
                                      const long long* offB_host, int* info, void* workspace,
                                      size_t workspace_bytes, int lane_max, int threads,
                                      bf_stream_t stream, bf_ragged_plan_t* plan);
int bf_ragged_plan_launch(bf_ragged_plan_t plan, bf_stream_t stream);
int bf_ragged_plan_info(bf_ragged_plan_t plan, int* out);
int bf_ragged_plan_destroy(bf_ragged_plan_t plan);

/* ------------------------------------------------------------------------ */
/* Allocation-free ragged solve (the paper has no counterpart).  For callers */
/* that cannot allocate device memory when they solve -- a controller whose */
/* memory is sized once at start-up and whose control loop may not allocate, */
/* or code that cannot hand the library a workspace -- this call runs the    */
/* same persistent kernel as the plan above, without a CUDA graph and        */
/* without any workspace: its queue lives in a file-scope device array of    */
/* BF_RAGGED_NOALLOC_MAX problems (about 0.77 MB), which every GPU that loads */
/* the library holds until the process exits.  Arguments are those of the    */
/* plan (no workspace); the call allocates nothing, on the device or on the  */
/* host.                                                                     */
/*  - batch > BF_RAGGED_NOALLOC_MAX returns BF_ERR_NOALLOC_LIMIT (nothing is */
/*    launched).                                                             */
/*  - The first call on a device looks up the array's device address (set-  */
/*    up); make that first call before any stream capture.  The address is   */
/*    kept for the process: do not call cudaDeviceReset on a device after    */
/*    using this entry point there.                                          */
/*  - The problem queue is copied to the array from host memory that the     */
/*    next call reuses, so a call on a stream that is being captured returns */
/*    BF_ERR_NOT_SUPPORTED and launches nothing.                             */
/*  - Every call shares the one array and overwrites it (the queue counter   */
/*    is cleared each call): calls that overlap on the GPU -- on different   */
/*    streams, or from different host threads -- race; serialise them, e.g. */
/*    on one stream.                                                         */
/* ------------------------------------------------------------------------ */
#define BF_RAGGED_NOALLOC_MAX 32768

int bf_ragged_potrf_potrs_noalloc(int batch, const int* n_host, int nrhs, double* S,
                                  const long long* offS_host, double* B,
                                  const long long* offB_host, int* info, int lane_max,
                                  int threads, bf_stream_t stream);

/* ------------------------------------------------------------------------ */
/* The size switch (section 2.4: the switch point between variants depends  */
/* on the routine and the architecture and is set by measurement).           */
/* bf_tune_set adds a table entry, consulted before the built-in defaults:    */
/*   routine  BF_ROUTINE_*                                                    */
/*   code     dgemm: 2*transA + transB; dtrsm: 8*right + 4*upper + 2*trans +  */
/*            unit; dpotrf: lda & 1 (even / odd leading dimension);       */
/*            dgetrf: 0 (entries hold only with BF_TUNE_FORCE).             */
/*            -1 matches every code.                                        */
/*   [n_lo, n_hi]  matrix order range (dgemm: max(m, n); dtrsm: order of A)   */
/*   variant  BF_VARIANT_*, optionally | BF_TUNE_FORCE                        */
/*   p0..p3   dgemm: TM, TN, KC, P (super-tile rows/cols, k-slice, problems   */
/*            per CTA; 0 = default); dtrsm: MR (4/8), P, CTAs per SM (1/2);  */
/*            dpotrf: T, NB,                                                */
/*            lane row-block height (4/8) or team size (2/4), lane k-loop   */
/*            unroll (1/2).                                                 */
/* Later entries take precedence.  bf_tune_clear removes all entries (and the */
/* batch rules below).                                                        */
/* bf_tune_query writes the configuration a call would use into out[5]:       */
/* {variant, p0, p1, p2, p3} in the order above (dgemm: variant,TM,TN,KC,P).  */
/* ------------------------------------------------------------------------ */
int bf_tune_set(int routine, int code, int n_lo, int n_hi, int variant, int p0, int p1, int p2,
                int p3);

/* The batch-size side of dpotrf's switch, set by measurement like the size side (section     */
/* 2.4).  For orders in [n_lo, n_hi] and lda parity `code` (-1: both), batches of at most     */
/* cta_max problems run one problem per CTA; larger ones up to team4_max run teams of 4 lanes */
/* per problem, then up to team2_max teams of 2; the rest take the table's variant.  A       */
/* negative cta_max keeps the built-in bound; negative team4_max and team2_max together keep  */
/* the built-in team bounds, and one negative alone means no team of that size.  Batches up   */
/* to the group form's built-in bound (BF_VARIANT_GROUP, orders 4..192) keep the group form:  */
/* a rule decides among the forms above it.  Entries with BF_TUNE_FORCE are not affected.     */
/* Later rules take precedence; bf_tune_clear removes them.  Returns 0, or minus the position */
/* of an illegal argument (routine other than BF_ROUTINE_DPOTRF: -1).                         */
int bf_tune_set_batch_rule(int routine, int code, int n_lo, int n_hi, long long cta_max,
                           long long team4_max, long long team2_max);
void bf_tune_clear(void);
int bf_tune_query(int routine, int code, int m, int n, int k, long long batch, int* out);

/* ------------------------------------------------------------------------ */
/* Measurement support (no counterpart in the paper).                        */
/* bf_launch_count: number of kernels this library has launched since it was */
/* loaded (host-side counter; differences over a region count its launches). */
/* bf_probe_fp64: launches `blocks` CTAs of 256 threads, each issuing        */
/* iters * 16 FP64 fused multiply-adds (2 flops each; a 4x4 register tile)   */
/* and writing                                                               */
/* one double per thread to out (device, blocks * 256 doubles).  Timed by    */
/* the caller, it measures the FP64 FMA throughput that bounds the routines. */
/* ------------------------------------------------------------------------ */
unsigned long long bf_launch_count(void);
int bf_probe_fp64(int blocks, int iters, double* out, bf_stream_t stream);
/* bf_probe_fp64_ex: the same measurement with `threads` per CTA (multiple of */
/* 32), only `active` lanes of each warp issuing (0..32; FP64 issue cost vs  */
/* lane mask), and chains = 0 (4x4 tile pattern, 16 FMAs per iteration) or 1 */
/* (one dependent chain a = fma(a, b, c), 16 per iteration).  out holds       */
/* blocks * threads doubles.                                                 */
int bf_probe_fp64_ex(int blocks, int threads, int iters, int active, int chains, double* out,
                     bf_stream_t stream);
/* bf_probe_kind: `blocks` CTAs of `threads` (multiple of 32) threads, every */
/* thread running `iters` iterations of one instruction kind; out holds      */
/* blocks * threads doubles.  Per iteration and warp:                        */
/*   kind 0  4 FP64 tensor-core MMAs mma.sync m8n8k4 (512 flops each)        */
/*   kind 1  4 FP64 tensor-core MMAs mma.sync m16n8k4 (1024 flops each)      */
/*   kind 2  per thread 4 x (FP64 sqrt + one FMA)                            */
/*   kind 3  per thread 4 x (FP64 1/x + one FMA)                             */
/*   kind 4  per thread 4 x (FP64 rsqrt + one FMA)                           */
/*   kind 5  per thread 16 binary32 FMAs (4x4 register tile)                 */
/*   kind 6  per thread 16 FP64 FMAs (4x4 tile), only in the warps whose     */
/*           index in the CTA is a multiple of 4 (the others exit at once)   */
/* Timed by the caller beside bf_probe_fp64_ex, it decides whether the FP64 */
/* tensor cores beat FP64 FMA (the routines' inner kernel, section 3.2) and  */
/* what a pivot's square root or reciprocal costs in FMA issue slots.        */
int bf_probe_kind(int kind, int blocks, int threads, int iters, double* out, bf_stream_t stream);

/* Human-readable text for a return code. */
const char* bf_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* BFGPU_H */
