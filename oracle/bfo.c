/*
 * bfo.c -- the CPU oracle: plain, slow, obviously correct FP64 definitions of
 * every operation the batched GPU library computes.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  The GPU library never
 * links, calls or includes it, and it shares no code with the GPU kernels.
 *
 * Storage: every matrix is column-major with a leading dimension, as in the
 * BLAS interface the paper keeps (section 2.1, "Notation": element (i,j) of a
 * matrix X with leading dimension ldx lives at X[i + j*ldx]).
 *
 * Arithmetic: IEEE binary64, evaluated in the natural loop order written
 * below.  The build uses -ffp-contract=off so that x86 and Arm hosts round
 * identically (no silent FMA contraction).
 *
 * Parity status: every exported function is pinned by tests that do not use
 * this file's arithmetic (closed forms, exact integer cases, brute-force
 * expansions, invariants, finite differences); see the test files named
 * test_oracle_*.py.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

static int is_n(char c) { return c == 'N' || c == 'n'; }
static int is_t(char c) { return c == 'T' || c == 't' || c == 'C' || c == 'c'; }
static int is_l(char c) { return c == 'L' || c == 'l'; }
static int is_u(char c) { return c == 'U' || c == 'u'; }
static int is_r(char c) { return c == 'R' || c == 'r'; }

int bfo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void bfo_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ------------------------------------------------------------------------ */
/* dgemm -- section 2.1: C <= alpha * op(A) * op(B) + beta * C, with C m x n   */
/* and k the length of each dot product.  op(X) = X for 'N', X^T for 'T'.    */
/* BLAS semantics the paper inherits: when beta == 0, C is written without   */
/* being read (so a NaN already in C does not propagate).                    */
/* ------------------------------------------------------------------------ */
int bfo_dgemm(char ta, char tb, int m, int n, int k, double alpha,
              const double* A, int lda, const double* B, int ldb,
              double beta, double* C, int ldc) {
    if (!(is_n(ta) || is_t(ta))) return -1;
    if (!(is_n(tb) || is_t(tb))) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 0) return -5;
    for (int j = 0; j < n; j++) {
        for (int i = 0; i < m; i++) {
            double s = 0.0;
            for (int p = 0; p < k; p++) {
                double a = is_n(ta) ? A[IDX(i, p, lda)] : A[IDX(p, i, lda)];
                double b = is_n(tb) ? B[IDX(p, j, ldb)] : B[IDX(j, p, ldb)];
                s += a * b;
            }
            double c = (beta == 0.0) ? 0.0 : beta * C[IDX(i, j, ldc)];
            C[IDX(i, j, ldc)] = alpha * s + c;
        }
    }
    return 0;
}

void bfo_dgemm_sb(char ta, char tb, int m, int n, int k, double alpha,
                  const double* A, int lda, long long sA,
                  const double* B, int ldb, long long sB, double beta,
                  double* C, int ldc, long long sC, int batch) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < batch; b++)
        bfo_dgemm(ta, tb, m, n, k, alpha, A + (size_t)b * sA, lda,
                  B + (size_t)b * sB, ldb, beta, C + (size_t)b * sC, ldc);
}

/* ------------------------------------------------------------------------ */
/* dpotrf, lower -- section 3.1 ("dpotrf"): A = L * L^T with L lower          */
/* triangular and a positive diagonal.  Unblocked textbook recurrence, for    */
/* j = 0..n-1:                                                               */
/*   d     = a_jj - sum_{p<j} l_jp^2                                         */
/*   l_jj  = sqrt(d)                   (fails when d <= 0 or d is NaN)        */
/*   l_ij  = (a_ij - sum_{p<j} l_ip l_jp) / l_jj     for i > j               */
/* Only the lower triangle is read and written; the strict upper triangle    */
/* and the rows beyond n in the leading dimension are never touched.         */
/* Returns LAPACK's info: 0 on success, j+1 (1-based) if the leading minor   */
/* of order j+1 is not positive definite; the factorisation stops there.     */
/* ------------------------------------------------------------------------ */
int bfo_dpotrf_l(int n, double* A, int lda) {
    for (int j = 0; j < n; j++) {
        double d = A[IDX(j, j, lda)];
        for (int p = 0; p < j; p++) d -= A[IDX(j, p, lda)] * A[IDX(j, p, lda)];
        if (!(d > 0.0)) {
            return j + 1;
        }
        double ljj = sqrt(d);
        A[IDX(j, j, lda)] = ljj;
        for (int i = j + 1; i < n; i++) {
            double s = A[IDX(i, j, lda)];
            for (int p = 0; p < j; p++) s -= A[IDX(i, p, lda)] * A[IDX(j, p, lda)];
            A[IDX(i, j, lda)] = s / ljj;
        }
    }
    return 0;
}

void bfo_dpotrf_l_sb(int n, double* A, int lda, long long sA, int batch, int* info) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < batch; b++) info[b] = bfo_dpotrf_l(n, A + (size_t)b * sA, lda);
}

/* ------------------------------------------------------------------------ */
/* dtrsm -- section 3.1 ("dtrsm"): triangular solve with the triangular      */
/* matrix A on the left (op(A) X = alpha B) or on the right                  */
/* (X op(A) = alpha B); X overwrites B (B is m x n).  uplo says which        */
/* triangle of A is stored, diag 'U' means a unit diagonal that is not read. */
/* Written from the definition: T = op(A) is lower or upper triangular, and  */
/* each case is a plain forward or backward substitution.  The oracle does   */
/* NOT use the paper's reduction of left solves to right solves by           */
/* transposition, so it stays independent of that design choice.            */
/* ------------------------------------------------------------------------ */
static double tri_elem(const double* A, int lda, int trans, int i, int j) {
    return trans ? A[IDX(j, i, lda)] : A[IDX(i, j, lda)];
}

int bfo_dtrsm(char side, char uplo, char ta, char diag, int m, int n, double alpha,
              const double* A, int lda, double* B, int ldb) {
    if (!(is_l(side) || is_r(side))) return -1;
    if (!(is_l(uplo) || is_u(uplo))) return -2;
    if (!(is_n(ta) || is_t(ta))) return -3;
    if (!(is_u(diag) || is_n(diag))) return -4;
    if (m < 0) return -5;
    if (n < 0) return -6;
    const int trans = is_t(ta);
    const int unit = is_u(diag);
    /* op(A) is lower triangular when (stored lower, no transpose) or (stored upper, transpose) */
    const int t_lower = (is_l(uplo) && !trans) || (is_u(uplo) && trans);
    if (is_l(side)) {
        /* T X = alpha B, T m x m; each column of B is an independent system */
        for (int c = 0; c < n; c++) {
            if (t_lower) {
                for (int i = 0; i < m; i++) {
                    double s = alpha * B[IDX(i, c, ldb)];
                    for (int p = 0; p < i; p++) s -= tri_elem(A, lda, trans, i, p) * B[IDX(p, c, ldb)];
                    B[IDX(i, c, ldb)] = unit ? s : s / tri_elem(A, lda, trans, i, i);
                }
            } else {
                for (int i = m - 1; i >= 0; i--) {
                    double s = alpha * B[IDX(i, c, ldb)];
                    for (int p = i + 1; p < m; p++) s -= tri_elem(A, lda, trans, i, p) * B[IDX(p, c, ldb)];
                    B[IDX(i, c, ldb)] = unit ? s : s / tri_elem(A, lda, trans, i, i);
                }
            }
        }
    } else {
        /* X T = alpha B, T n x n; each row of B is an independent system:   */
        /* sum_p x_rp T_pj = alpha b_rj                                      */
        for (int r = 0; r < m; r++) {
            if (t_lower) {
                /* T_pj != 0 only for p >= j: solve j = n-1 down to 0 */
                for (int j = n - 1; j >= 0; j--) {
                    double s = alpha * B[IDX(r, j, ldb)];
                    for (int p = j + 1; p < n; p++) s -= B[IDX(r, p, ldb)] * tri_elem(A, lda, trans, p, j);
                    B[IDX(r, j, ldb)] = unit ? s : s / tri_elem(A, lda, trans, j, j);
                }
            } else {
                /* T_pj != 0 only for p <= j: solve j = 0 up to n-1 */
                for (int j = 0; j < n; j++) {
                    double s = alpha * B[IDX(r, j, ldb)];
                    for (int p = 0; p < j; p++) s -= B[IDX(r, p, ldb)] * tri_elem(A, lda, trans, p, j);
                    B[IDX(r, j, ldb)] = unit ? s : s / tri_elem(A, lda, trans, j, j);
                }
            }
        }
    }
    return 0;
}

void bfo_dtrsm_sb(char side, char uplo, char ta, char diag, int m, int n, double alpha,
                  const double* A, int lda, long long sA, double* B, int ldb, long long sB,
                  int batch) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < batch; b++)
        bfo_dtrsm(side, uplo, ta, diag, m, n, alpha, A + (size_t)b * sA, lda,
                  B + (size_t)b * sB, ldb);
}

/* ------------------------------------------------------------------------ */
/* dpotrs, lower: given the factor L of A = L L^T, solve A X = B in two      */
/* substitutions, Y = L^{-1} B (forward) then X = L^{-T} Y (backward).        */
/* This is the solve that follows dpotrf in section 5's command tables       */
/* (back/forward-slash with an SPD matrix).                                  */
/* ------------------------------------------------------------------------ */
void bfo_dpotrs_l(int n, int nrhs, const double* L, int ldl, double* B, int ldb) {
    for (int c = 0; c < nrhs; c++) {
        double* b = B + (size_t)c * ldb;
        for (int i = 0; i < n; i++) {
            double s = b[i];
            for (int p = 0; p < i; p++) s -= L[IDX(i, p, ldl)] * b[p];
            b[i] = s / L[IDX(i, i, ldl)];
        }
        for (int i = n - 1; i >= 0; i--) {
            double s = b[i];
            for (int p = i + 1; p < n; p++) s -= L[IDX(p, i, ldl)] * b[p];
            b[i] = s / L[IDX(i, i, ldl)];
        }
    }
}

void bfo_dpotrs_l_sb(int n, int nrhs, const double* L, int ldl, long long sL,
                     double* B, int ldb, long long sB, int batch) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < batch; b++)
        bfo_dpotrs_l(n, nrhs, L + (size_t)b * sL, ldl, B + (size_t)b * sB, ldb);
}

/* ------------------------------------------------------------------------ */
/* Ragged batch: problem b has its own order n[b]; its SPD matrix (leading   */
/* dimension n[b]) starts at S + offS[b] and its n[b] x nrhs right-hand      */
/* sides (leading dimension n[b]) at X + offX[b].  Each problem is factored  */
/* in place (dpotrf, lower) and, when info == 0, solved in place (dpotrs).   */
/* ------------------------------------------------------------------------ */
void bfo_ragged_potrf_potrs(int batch, const int* n, const long long* offS, double* S,
                            const long long* offX, double* X, int nrhs, int* info) {
    #pragma omp parallel for schedule(dynamic, 8)
    for (int b = 0; b < batch; b++) {
        double* Sb = S + offS[b];
        info[b] = bfo_dpotrf_l(n[b], Sb, n[b]);
        if (info[b] == 0) bfo_dpotrs_l(n[b], nrhs, Sb, n[b], X + offX[b], n[b]);
    }
}

/* ------------------------------------------------------------------------ */
/* Normwise backward error of an approximate solution x of A x = b          */
/* (Rigal & Gaches):  eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) */
/* with the residual formed in FP64.  A is a full (symmetric) n x n matrix.  */
/* ------------------------------------------------------------------------ */
double bfo_backward_error(int n, const double* A, int lda, const double* x, const double* b) {
    double rnorm = 0.0, anorm = 0.0, xnorm = 0.0, bnorm = 0.0;
    for (int i = 0; i < n; i++) {
        double r = b[i], arow = 0.0;
        for (int j = 0; j < n; j++) {
            r -= A[IDX(i, j, lda)] * x[j];
            arow += fabs(A[IDX(i, j, lda)]);
        }
        if (fabs(r) > rnorm) rnorm = fabs(r);
        if (arow > anorm) anorm = arow;
        if (fabs(x[i]) > xnorm) xnorm = fabs(x[i]);
        if (fabs(b[i]) > bnorm) bnorm = fabs(b[i]);
    }
    double den = anorm * xnorm + bnorm;
    return den > 0.0 ? rnorm / den : rnorm;
}

void bfo_backward_error_sb(int n, const double* A, int lda, long long sA, const double* x,
                           long long sx, const double* b, long long sb, int batch, double* eta) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int p = 0; p < batch; p++)
        eta[p] = bfo_backward_error(n, A + (size_t)p * sA, lda, x + (size_t)p * sx, b + (size_t)p * sb);
}

/* ------------------------------------------------------------------------ */
/* Mixed-precision SPD solve (single right-hand side), the refined form:     */
/*   1. round A to binary32 and factor it A32 = L32 L32^T with the same      */
/*      unblocked recurrence as bfo_dpotrf_l, in binary32, except that each  */
/*      pivot d is tested for positivity and square-rooted in binary64       */
/*      before being rounded to binary32;                                    */
/*   2. x = L32^{-T} L32^{-1} b   (binary32 substitutions, x kept in FP64);   */
/*   3. repeat: r = b - A x in binary64; stop when eta(x) <= tol;            */
/*      d = L32^{-T} L32^{-1} r (binary32); x = x + d in binary64.           */
/* If the binary32 factorisation fails, or the iteration cap is reached      */
/* without convergence, the problem is solved in binary64 (dpotrf+dpotrs)    */
/* and flagged, as LAPACK's dsposv does.  Returns the number of refinement   */
/* steps taken (0 = the first solution already met tol), or -1 when it fell  */
/* back to binary64; *info is the binary64 dpotrf info in the fallback case. */
/* ------------------------------------------------------------------------ */
static int spotrf_l_f64piv(int n, float* L, int ld) {
    for (int j = 0; j < n; j++) {
        float d = L[IDX(j, j, ld)];
        for (int p = 0; p < j; p++) d -= L[IDX(j, p, ld)] * L[IDX(j, p, ld)];
        double dd = (double)d;
        if (!(dd > 0.0)) return j + 1;
        float ljj = (float)sqrt(dd);
        L[IDX(j, j, ld)] = ljj;
        for (int i = j + 1; i < n; i++) {
            float s = L[IDX(i, j, ld)];
            for (int p = 0; p < j; p++) s -= L[IDX(i, p, ld)] * L[IDX(j, p, ld)];
            L[IDX(i, j, ld)] = s / ljj;
        }
    }
    return 0;
}

static void spotrs_l(int n, const float* L, int ld, float* b) {
    for (int i = 0; i < n; i++) {
        float s = b[i];
        for (int p = 0; p < i; p++) s -= L[IDX(i, p, ld)] * b[p];
        b[i] = s / L[IDX(i, i, ld)];
    }
    for (int i = n - 1; i >= 0; i--) {
        float s = b[i];
        for (int p = i + 1; p < n; p++) s -= L[IDX(p, i, ld)] * b[p];
        b[i] = s / L[IDX(i, i, ld)];
    }
}

int bfo_dsposv(int n, const double* A, int lda, const double* b, double* x,
               double tol, int itmax, int* info) {
    *info = 0;
    float* L = (float*)malloc(sizeof(float) * (size_t)n * (size_t)n + sizeof(float) * (size_t)n);
    float* w = L + (size_t)n * n;
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) L[IDX(i, j, n)] = (float)A[IDX(i, j, lda)];
    int iters = -1;
    if (spotrf_l_f64piv(n, L, n) == 0) {
        for (int i = 0; i < n; i++) w[i] = (float)b[i];
        spotrs_l(n, L, n, w);
        for (int i = 0; i < n; i++) x[i] = (double)w[i];
        for (int it = 0; it <= itmax; it++) {
            if (bfo_backward_error(n, A, lda, x, b) <= tol) { iters = it; break; }
            if (it == itmax) break;
            for (int i = 0; i < n; i++) {
                double s = b[i];
                for (int j = 0; j < n; j++) s -= A[IDX(i, j, lda)] * x[j];
                r[i] = s;
            }
            for (int i = 0; i < n; i++) w[i] = (float)r[i];
            spotrs_l(n, L, n, w);
            for (int i = 0; i < n; i++) x[i] += (double)w[i];
        }
    }
    if (iters < 0) {
        double* F = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) F[IDX(i, j, n)] = A[IDX(i, j, lda)];
        *info = bfo_dpotrf_l(n, F, n);
        for (int i = 0; i < n; i++) x[i] = b[i];
        if (*info == 0) bfo_dpotrs_l(n, 1, F, n, x, n);
        free(F);
    }
    free(L);
    free(r);
    return iters;
}

void bfo_dsposv_sb(int n, const double* A, int lda, long long sA, const double* b, long long sb,
                   double* x, long long sx, double tol, int itmax, int batch, int* iters, int* info) {
    #pragma omp parallel for schedule(dynamic, 4)
    for (int p = 0; p < batch; p++)
        iters[p] = bfo_dsposv(n, A + (size_t)p * sA, lda, b + (size_t)p * sb, x + (size_t)p * sx,
                              tol, itmax, info + p);
}

/* ------------------------------------------------------------------------ */
/* Reverse mode of the unblocked Cholesky loop above.  Given L (the factor   */
/* of A, lower triangle) and Lbar = d(loss)/dL (lower triangle), returns     */
/* Abar_tril = d(loss)/dA with respect to the entries a_ij, i >= j, that the */
/* forward loop reads (the strict upper part of Abar is set to zero).        */
/* Each forward statement is reversed in the opposite order:                 */
/*   forward  l_ij = s_ij / l_jj,  s_ij = a_ij - sum_{p<j} l_ip l_jp (i > j)  */
/*            l_jj = sqrt(d_j),    d_j  = a_jj - sum_{p<j} l_jp^2            */
/*   reverse  sbar = lbar_ij / l_jj;  lbar_jj -= lbar_ij l_ij / l_jj;         */
/*            abar_ij = sbar;  lbar_ip -= sbar l_jp;  lbar_jp -= sbar l_ip    */
/*            dbar = lbar_jj / (2 l_jj); abar_jj = dbar; lbar_jp -= 2 dbar l_jp */
/* The symmetric gradient G (G = G^T, dloss = sum_ij G_ij dA_ij for a        */
/* symmetric perturbation) follows as G_ii = Abar_ii, G_ij = G_ji = Abar_ij/2.*/
/* ------------------------------------------------------------------------ */
void bfo_dpotrf_l_adjoint(int n, const double* L, int ldl, const double* Lbar, int ldlb,
                          double* Abar, int ldab) {
    double* lb = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) lb[IDX(i, j, n)] = (i >= j) ? Lbar[IDX(i, j, ldlb)] : 0.0;
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) Abar[IDX(i, j, ldab)] = 0.0;
    for (int j = n - 1; j >= 0; j--) {
        double ljj = L[IDX(j, j, ldl)];
        for (int i = n - 1; i > j; i--) {
            double sbar = lb[IDX(i, j, n)] / ljj;
            lb[IDX(j, j, n)] -= lb[IDX(i, j, n)] * L[IDX(i, j, ldl)] / ljj;
            Abar[IDX(i, j, ldab)] = sbar;
            for (int p = j - 1; p >= 0; p--) {
                lb[IDX(i, p, n)] -= sbar * L[IDX(j, p, ldl)];
                lb[IDX(j, p, n)] -= sbar * L[IDX(i, p, ldl)];
            }
        }
        double dbar = lb[IDX(j, j, n)] / (2.0 * ljj);
        Abar[IDX(j, j, ldab)] = dbar;
        for (int p = j - 1; p >= 0; p--) lb[IDX(j, p, n)] -= 2.0 * dbar * L[IDX(j, p, ldl)];
    }
    free(lb);
}

/* ------------------------------------------------------------------------ */
/* Closed-form gradient of the SPD-solve loss used by the differentiation    */
/* workload, which avoids differentiating through the Cholesky at all:       */
/*   A = Q + J J^T (Q diagonal, J n x q), X = A^{-1} B (B n x r),            */
/*   loss = sum_ij X_ij W_ij.                                                */
/*   Y = A^{-1} W,  Bbar = Y,  Wbar = X,                                     */
/*   G = -(Y X^T + X Y^T)/2  (symmetric gradient with respect to A),          */
/*   Jbar = 2 G J,  qbar_i = G_ii.                                           */
/* The two solves use the oracle's own dpotrf + dpotrs.  Returns dpotrf info.*/
/* All matrices have leading dimension equal to their row count.             */
/* ------------------------------------------------------------------------ */
int bfo_spd_solve_loss_grad(int n, int q, int r, const double* Qd, const double* J,
                            const double* B, const double* W, double* X, double* loss,
                            double* Jbar, double* Qbar, double* Bbar, double* Wbar) {
    double* A = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* G = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* Y = (double*)malloc(sizeof(double) * (size_t)n * r);
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) A[IDX(i, j, n)] = (i == j) ? Qd[i] : 0.0;
    bfo_dgemm('N', 'T', n, n, q, 1.0, J, n, J, n, 1.0, A, n);
    int info = bfo_dpotrf_l(n, A, n);
    if (info == 0) {
        memcpy(X, B, sizeof(double) * (size_t)n * r);
        bfo_dpotrs_l(n, r, A, n, X, n);
        memcpy(Y, W, sizeof(double) * (size_t)n * r);
        bfo_dpotrs_l(n, r, A, n, Y, n);
        double l = 0.0;
        for (size_t e = 0; e < (size_t)n * r; e++) l += X[e] * W[e];
        *loss = l;
        /* G = -(Y X^T + X Y^T) / 2 */
        bfo_dgemm('N', 'T', n, n, r, -0.5, Y, n, X, n, 0.0, G, n);
        bfo_dgemm('N', 'T', n, n, r, -0.5, X, n, Y, n, 1.0, G, n);
        bfo_dgemm('N', 'N', n, q, n, 2.0, G, n, J, n, 0.0, Jbar, n);
        for (int i = 0; i < n; i++) Qbar[i] = G[IDX(i, i, n)];
        memcpy(Bbar, Y, sizeof(double) * (size_t)n * r);
        memcpy(Wbar, X, sizeof(double) * (size_t)n * r);
    }
    free(A);
    free(G);
    free(Y);
    return info;
}

void bfo_spd_solve_loss_grad_sb(int n, int q, int r, int batch, const double* Qd, const double* J,
                                const double* B, const double* W, double* X, double* loss,
                                double* Jbar, double* Qbar, double* Bbar, double* Wbar, int* info) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int p = 0; p < batch; p++) {
        size_t nq = (size_t)n * q, nr = (size_t)n * r;
        info[p] = bfo_spd_solve_loss_grad(n, q, r, Qd + (size_t)p * n, J + p * nq, B + p * nr,
                                          W + p * nr, X + p * nr, loss + p, Jbar + p * nq,
                                          Qbar + (size_t)p * n, Bbar + p * nr, Wbar + p * nr);
    }
}

/* ------------------------------------------------------------------------ */
/* dsyrk -- section 3.1 ("dsyrk": dgemm whose A and B coincide):            */
/*   C <= alpha * op(A) * op(A)^T + beta * C,  C n x n symmetric,            */
/* op(A) = A (n x k) for trans 'N', A^T (A stored k x n) for 'T'.  Only the  */
/* uplo triangle of C is read and written.  BLAS semantics: beta == 0       */
/* writes without reading C; alpha == 0 does not read A.                     */
/* ------------------------------------------------------------------------ */
static double opa(const double* A, int lda, int tr, int i, int p) {
    return tr ? A[IDX(p, i, lda)] : A[IDX(i, p, lda)];
}

int bfo_dsyrk(char uplo, char trans, int n, int k, double alpha, const double* A, int lda,
              double beta, double* C, int ldc) {
    if (!(is_l(uplo) || is_u(uplo))) return -1;
    if (!(is_n(trans) || is_t(trans))) return -2;
    if (n < 0) return -3;
    if (k < 0) return -4;
    const int tr = is_t(trans);
    if (lda < ((tr ? k : n) > 1 ? (tr ? k : n) : 1)) return -7;
    if (ldc < (n > 1 ? n : 1)) return -10;
    if (n == 0 || ((alpha == 0.0 || k == 0) && beta == 1.0)) return 0;
    const int low = is_l(uplo);
    for (int j = 0; j < n; j++) {
        const int i0 = low ? j : 0, i1 = low ? n : j + 1;
        for (int i = i0; i < i1; i++) {
            double s = 0.0;
            if (alpha != 0.0)
                for (int p = 0; p < k; p++) s += opa(A, lda, tr, i, p) * opa(A, lda, tr, j, p);
            C[IDX(i, j, ldc)] = (beta == 0.0) ? alpha * s : alpha * s + beta * C[IDX(i, j, ldc)];
        }
    }
    return 0;
}

void bfo_dsyrk_sb(char uplo, char trans, int n, int k, double alpha, const double* A, int lda,
                  long long sA, double beta, double* C, int ldc, long long sC, int batch) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < batch; b++)
        bfo_dsyrk(uplo, trans, n, k, alpha, A + (size_t)b * sA, lda, beta, C + (size_t)b * sC, ldc);
}

/* ------------------------------------------------------------------------ */
/* dsyrk followed by dpotrf, lower: C <= chol(C + A * A^T), A n x k -- the  */
/* fused routine of the paper's own API that section 5 credits for part of  */
/* the Riccati recursion's speed-up.  Defined as the two calls in sequence;  */
/* returns dpotrf's info.                                                    */
/* ------------------------------------------------------------------------ */
int bfo_dsyrk_dpotrf_l(int n, int k, const double* A, int lda, double* C, int ldc) {
    bfo_dsyrk('L', 'N', n, k, 1.0, A, lda, 1.0, C, ldc);
    return bfo_dpotrf_l(n, C, ldc);
}

void bfo_dsyrk_dpotrf_l_sb(int n, int k, const double* A, int lda, long long sA, double* C, int ldc,
                           long long sC, int batch, int* info) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < batch; b++)
        info[b] = bfo_dsyrk_dpotrf_l(n, k, A + (size_t)b * sA, lda, C + (size_t)b * sC, ldc);
}

/* ------------------------------------------------------------------------ */
/* dtrmm -- section 3.1 ("dtrmm", treated like dtrsm) and the Riccati        */
/* recursion of section 5 (dtrmm_rlnn): B <= alpha * op(A) * B (side 'L', A  */
/* m x m) or B <= alpha * B * op(A) (side 'R', A n x n).  uplo: the stored   */
/* triangle of A; diag 'U': unit diagonal, not read.  Written from the       */
/* definition: T = op(A) is made explicit (zero outside its triangle), the   */
/* product is formed in a temporary with plain loops, then scaled into B.    */
/* alpha == 0 sets B to zero without reading A or B (BLAS).                  */
/* ------------------------------------------------------------------------ */
int bfo_dtrmm(char side, char uplo, char ta, char diag, int m, int n, double alpha,
              const double* A, int lda, double* B, int ldb) {
    if (!(is_l(side) || is_r(side))) return -1;
    if (!(is_l(uplo) || is_u(uplo))) return -2;
    if (!(is_n(ta) || is_t(ta))) return -3;
    if (!(is_u(diag) || is_n(diag))) return -4;
    if (m < 0) return -5;
    if (n < 0) return -6;
    if (m == 0 || n == 0) return 0;
    if (alpha == 0.0) {
        for (int j = 0; j < n; j++)
            for (int i = 0; i < m; i++) B[IDX(i, j, ldb)] = 0.0;
        return 0;
    }
    const int left = is_l(side), trans = is_t(ta), unit = is_u(diag);
    const int k = left ? m : n;
    const int t_lower = (is_l(uplo) && !trans) || (is_u(uplo) && trans);
    double* T = (double*)calloc((size_t)k * k, sizeof(double));
    double* R = (double*)malloc(sizeof(double) * (size_t)m * n);
    for (int j = 0; j < k; j++)
        for (int i = 0; i < k; i++) {
            if (i == j) T[IDX(i, j, k)] = unit ? 1.0 : tri_elem(A, lda, trans, i, i);
            else if (t_lower ? (i > j) : (i < j)) T[IDX(i, j, k)] = tri_elem(A, lda, trans, i, j);
        }
    for (int j = 0; j < n; j++)
        for (int i = 0; i < m; i++) {
            double s = 0.0;
            if (left)
                for (int p = 0; p < m; p++) s += T[IDX(i, p, k)] * B[IDX(p, j, ldb)];
            else
                for (int p = 0; p < n; p++) s += B[IDX(i, p, ldb)] * T[IDX(p, j, k)];
            R[IDX(i, j, m)] = s;
        }
    for (int j = 0; j < n; j++)
        for (int i = 0; i < m; i++) B[IDX(i, j, ldb)] = alpha * R[IDX(i, j, m)];
    free(T);
    free(R);
    return 0;
}

void bfo_dtrmm_sb(char side, char uplo, char ta, char diag, int m, int n, double alpha,
                  const double* A, int lda, long long sA, double* B, int ldb, long long sB,
                  int batch) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < batch; b++)
        bfo_dtrmm(side, uplo, ta, diag, m, n, alpha, A + (size_t)b * sA, lda, B + (size_t)b * sB, ldb);
}

/* ------------------------------------------------------------------------ */
/* dpotrf, upper -- appendix table of LAPACK routines (dpotrf_u, chol(Q,    */
/* 'upper')): A = U^T U with U upper triangular, positive diagonal.          */
/* Unblocked recurrence on the upper triangle, for j = 0..n-1:               */
/*   d     = a_jj - sum_{p<j} u_pj^2,  u_jj = sqrt(d)  (fails: d <= 0 / NaN)   */
/*   u_ji  = (a_ji - sum_{p<j} u_pj u_pi) / u_jj     for i > j               */
/* Only the upper triangle is read and written.  LAPACK info as dpotrf_l.    */
/* ------------------------------------------------------------------------ */
int bfo_dpotrf_u(int n, double* A, int lda) {
    for (int j = 0; j < n; j++) {
        double d = A[IDX(j, j, lda)];
        for (int p = 0; p < j; p++) d -= A[IDX(p, j, lda)] * A[IDX(p, j, lda)];
        if (!(d > 0.0)) return j + 1;
        const double ujj = sqrt(d);
        A[IDX(j, j, lda)] = ujj;
        for (int i = j + 1; i < n; i++) {
            double s = A[IDX(j, i, lda)];
            for (int p = 0; p < j; p++) s -= A[IDX(p, j, lda)] * A[IDX(p, i, lda)];
            A[IDX(j, i, lda)] = s / ujj;
        }
    }
    return 0;
}

void bfo_dpotrf_u_sb(int n, double* A, int lda, long long sA, int batch, int* info) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < batch; b++) info[b] = bfo_dpotrf_u(n, A + (size_t)b * sA, lda);
}

/* ------------------------------------------------------------------------ */
/* dgetrf -- section 3.1 ("dgetrf"): LU factorisation with partial (row)     */
/* pivoting, P A = L U, A m x n, L unit lower (stored below the diagonal),   */
/* U upper.  Unblocked, column by column, for j = 0..min(m,n)-1:             */
/*   p = the first row index i >= j of the largest |a_ij| (a NaN never      */
/*       counts as larger);  ipiv[j] = p + 1 (1-based, as LAPACK);           */
/*   if a_pj != 0: swap rows j and p across all n columns, then              */
/*       l_ij = a_ij / a_jj for i > j;                                       */
/*   else: info = j + 1 if it is the first zero pivot (the column is left);  */
/*   a_ik -= l_ij a_jk for i > j, k > j.                                     */
/* Returns info (0, or the 1-based column of the first exactly zero pivot:   */
/* U is then singular; the factorisation is still completed).                */
/* ------------------------------------------------------------------------ */
int bfo_dgetrf(int m, int n, double* A, int lda, int* ipiv) {
    int info = 0;
    const int mn = m < n ? m : n;
    for (int j = 0; j < mn; j++) {
        int p = j;
        double best = fabs(A[IDX(j, j, lda)]);
        for (int i = j + 1; i < m; i++) {
            const double v = fabs(A[IDX(i, j, lda)]);
            if (v > best) {
                best = v;
                p = i;
            }
        }
        ipiv[j] = p + 1;
        if (A[IDX(p, j, lda)] != 0.0) {
            if (p != j)
                for (int c = 0; c < n; c++) {
                    const double t = A[IDX(j, c, lda)];
                    A[IDX(j, c, lda)] = A[IDX(p, c, lda)];
                    A[IDX(p, c, lda)] = t;
                }
            for (int i = j + 1; i < m; i++) A[IDX(i, j, lda)] = A[IDX(i, j, lda)] / A[IDX(j, j, lda)];
        } else if (info == 0) {
            info = j + 1;
        }
        for (int c = j + 1; c < n; c++)
            for (int i = j + 1; i < m; i++) A[IDX(i, c, lda)] -= A[IDX(i, j, lda)] * A[IDX(j, c, lda)];
    }
    return info;
}

void bfo_dgetrf_sb(int m, int n, double* A, int lda, long long sA, int* ipiv, int batch, int* info) {
    const int mn = m < n ? m : n;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < batch; b++) info[b] = bfo_dgetrf(m, n, A + (size_t)b * sA, lda, ipiv + (size_t)b * mn);
}

/* ------------------------------------------------------------------------ */
/* dgetrs -- solve op(A) X = B with the factors of dgetrf (n x n):           */
/*   'N': B <- P B (the row swaps j <-> ipiv[j]-1, j ascending), then        */
/*        L Y = B (unit lower, forward), U X = Y (backward);                 */
/*   'T': U^T Y = B (forward), L^T Z = Y (unit, backward), then the swaps    */
/*        in descending order.                                              */
/* ------------------------------------------------------------------------ */
int bfo_dgetrs(char trans, int n, int nrhs, const double* A, int lda, const int* ipiv, double* B, int ldb) {
    if (!(is_n(trans) || is_t(trans))) return -1;
    for (int c = 0; c < nrhs; c++) {
        double* b = B + (size_t)c * ldb;
        if (is_n(trans)) {
            for (int j = 0; j < n; j++) {
                const int p = ipiv[j] - 1;
                if (p != j) {
                    const double t = b[j];
                    b[j] = b[p];
                    b[p] = t;
                }
            }
            for (int i = 0; i < n; i++) {
                double s = b[i];
                for (int p = 0; p < i; p++) s -= A[IDX(i, p, lda)] * b[p];
                b[i] = s;
            }
            for (int i = n - 1; i >= 0; i--) {
                double s = b[i];
                for (int p = i + 1; p < n; p++) s -= A[IDX(i, p, lda)] * b[p];
                b[i] = s / A[IDX(i, i, lda)];
            }
        } else {
            for (int i = 0; i < n; i++) {
                double s = b[i];
                for (int p = 0; p < i; p++) s -= A[IDX(p, i, lda)] * b[p];
                b[i] = s / A[IDX(i, i, lda)];
            }
            for (int i = n - 1; i >= 0; i--) {
                double s = b[i];
                for (int p = i + 1; p < n; p++) s -= A[IDX(p, i, lda)] * b[p];
                b[i] = s;
            }
            for (int j = n - 1; j >= 0; j--) {
                const int p = ipiv[j] - 1;
                if (p != j) {
                    const double t = b[j];
                    b[j] = b[p];
                    b[p] = t;
                }
            }
        }
    }
    return 0;
}

void bfo_dgetrs_sb(char trans, int n, int nrhs, const double* A, int lda, long long sA, const int* ipiv,
                   double* B, int ldb, long long sB, int batch) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < batch; b++)
        bfo_dgetrs(trans, n, nrhs, A + (size_t)b * sA, lda, ipiv + (size_t)b * n, B + (size_t)b * sB, ldb);
}

/* ------------------------------------------------------------------------ */
/* Riccati recursion, square-root form (section 5, "Riccati recursion"):    */
/* N stages, n_x states, n_u controls.  Inputs per stage s = 0..N-1:        */
/*   BAt_s = [B_s^T; A_s^T]  ((n_u+n_x) x n_x, column-major),               */
/*   RSQ_s = [R_s S_s; S_s^T Q_s]  ((n_u+n_x) square, SPD, lower read),      */
/* and the terminal Q_N (n_x x n_x, SPD).  With Lc_N = chol(Q_N), for        */
/* s = N-1 down to 0:                                                        */
/*   C   = BAt_s * Lc_{s+1}                      (dtrmm_rlnn)                */
/*   F_s = chol(RSQ_s + C C^T)                   (dsyrk_ln, then dpotrf_l)    */
/*   Lc_s = the trailing n_x x n_x block of F_s                              */
/* F (N+1 factors: F_s for s < N, then chol(Q_N) in the top-left n_x block   */
/* of F_N) receives every factor; returns 0 or the first failing stage's     */
/* dpotrf info + 1000 * stage.                                               */
/* ------------------------------------------------------------------------ */
int bfo_riccati(int N, int nx, int nu, const double* BAt, const double* RSQ, const double* QN, double* F) {
    const int m = nx + nu;
    const size_t fsz = (size_t)m * m;
    double* C = (double*)malloc(sizeof(double) * (size_t)m * nx);
    double* FN = F + (size_t)N * fsz;
    for (size_t e = 0; e < fsz; e++) FN[e] = 0.0;
    for (int j = 0; j < nx; j++)
        for (int i = 0; i < nx; i++) FN[IDX(i, j, m)] = QN[IDX(i, j, nx)];
    int info = bfo_dpotrf_l(nx, FN, m);
    if (info) {
        free(C);
        return info + 1000 * N;
    }
    const double* Lc = FN;  /* leading dimension m; chol(Q_N) sits at offset 0 */
    for (int s = N - 1; s >= 0; s--) {
        const double* Bs = BAt + (size_t)s * m * nx;
        double* Fs = F + (size_t)s * fsz;
        memcpy(C, Bs, sizeof(double) * (size_t)m * nx);
        /* dtrmm_rlnn on a copy of Lc with leading dimension nx */
        double* L = (double*)malloc(sizeof(double) * (size_t)nx * nx);
        for (int j = 0; j < nx; j++)
            for (int i = 0; i < nx; i++) L[IDX(i, j, nx)] = (i >= j) ? Lc[IDX(i, j, m)] : 0.0;
        bfo_dtrmm('R', 'L', 'N', 'N', m, nx, 1.0, L, nx, C, m);
        free(L);
        memcpy(Fs, RSQ + (size_t)s * fsz, sizeof(double) * fsz);
        info = bfo_dsyrk_dpotrf_l(m, nx, C, m, Fs, m);
        if (info) {
            free(C);
            return info + 1000 * s;
        }
        Lc = Fs + IDX(nu, nu, m);
    }
    free(C);
    return 0;
}

void bfo_riccati_sb(int N, int nx, int nu, const double* BAt, const double* RSQ, const double* QN, double* F,
                    int batch, int* info) {
    const int m = nx + nu;
    const size_t sB = (size_t)N * m * nx, sR = (size_t)N * m * m, sQ = (size_t)nx * nx, sF = (size_t)(N + 1) * m * m;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int b = 0; b < batch; b++)
        info[b] = bfo_riccati(N, nx, nu, BAt + b * sB, RSQ + b * sR, QN + b * sQ, F + b * sF);
}
