// bf_api.cu -- the extern "C" entry points of include/bfgpu.h: argument
// checking (LAPACK's negative-info rule), the size switch, and launch.
#include "bf_internal.h"
#include "../../include/bfgpu.h"

using namespace bf;

namespace {

inline bool is_n(char c) { return c == 'N' || c == 'n'; }
inline bool is_t(char c) { return c == 'T' || c == 't' || c == 'C' || c == 'c'; }
inline bool is_l(char c) { return c == 'L' || c == 'l'; }
inline bool is_u(char c) { return c == 'U' || c == 'u'; }
inline bool is_r(char c) { return c == 'R' || c == 'r'; }
inline int imax1(int a) { return a > 1 ? a : 1; }

inline int status(cudaError_t e) { return e == cudaSuccess ? BF_SUCCESS : BF_ERR_CUDA; }

// dgemm argument check; `pos` maps the logical argument to its 1-based position.
struct GemmPos {
    int ta, tb, m, n, k, A, lda, B, ldb, C, ldc, sC, batch;
};

int check_gemm(char ta, char tb, int m, int n, int k, const void* A, int lda, const void* B, int ldb,
               const void* C, int ldc, long long strideC, int batch, double alpha, double beta,
               const GemmPos& pos) {
    if (!(is_n(ta) || is_t(ta))) return -pos.ta;
    if (!(is_n(tb) || is_t(tb))) return -pos.tb;
    if (m < 0) return -pos.m;
    if (n < 0) return -pos.n;
    if (k < 0) return -pos.k;
    const int rowsA = is_n(ta) ? m : k;
    const int rowsB = is_n(tb) ? k : n;
    if (lda < imax1(rowsA)) return -pos.lda;
    if (ldb < imax1(rowsB)) return -pos.ldb;
    if (ldc < imax1(m)) return -pos.ldc;
    if (pos.batch && batch < 0) return -pos.batch;
    if (pos.sC && batch > 1 && strideC < (long long)ldc * n) return -pos.sC;
    const bool work = m > 0 && n > 0 && batch != 0;
    const bool readsAB = work && k > 0 && alpha != 0.0;
    if (readsAB && !A) return -pos.A;
    if (readsAB && !B) return -pos.B;
    if (work && !C) return -pos.C;
    (void)beta;
    return 0;
}

int run_gemm(char ta, char tb, int m, int n, int k, double alpha, MatRef A, int lda, MatRef B, int ldb,
             double beta, MatRef C, int ldc, long long batch, cudaStream_t s) {
    if (m == 0 || n == 0 || batch == 0) return 0;
    if ((alpha == 0.0 || k == 0) && beta == 1.0) return 0;
    const bool a = is_t(ta), b = is_t(tb);
    GemmConfig cfg = choose_gemm(a, b, m, n, k, lda, batch);
    return status(launch_dgemm(a, b, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, batch, cfg, 0,
                               nullptr, s));
}

struct TrsmPos {
    int side, uplo, ta, diag, m, n, A, lda, B, ldb, sB, batch;
};

int check_trsm(char side, char uplo, char ta, char diag, int m, int n, const void* A, int lda,
               const void* B, int ldb, long long strideB, int batch, double alpha, const TrsmPos& pos) {
    if (!(is_l(side) || is_r(side))) return -pos.side;
    if (!(is_l(uplo) || is_u(uplo))) return -pos.uplo;
    if (!(is_n(ta) || is_t(ta))) return -pos.ta;
    if (!(is_u(diag) || is_n(diag))) return -pos.diag;
    if (m < 0) return -pos.m;
    if (n < 0) return -pos.n;
    const int order = is_l(side) ? m : n;
    if (lda < imax1(order)) return -pos.lda;
    if (ldb < imax1(m)) return -pos.ldb;
    if (pos.batch && batch < 0) return -pos.batch;
    if (pos.sB && batch > 1 && strideB < (long long)ldb * n) return -pos.sB;
    const bool work = m > 0 && n > 0 && batch != 0;
    if (work && alpha != 0.0 && !A) return -pos.A;
    if (work && !B) return -pos.B;
    return 0;
}

int run_trsm(char side, char uplo, char ta, char diag, int m, int n, double alpha, MatRef A, int lda,
             MatRef B, int ldb, long long batch, cudaStream_t s) {
    if (m == 0 || n == 0 || batch == 0) return 0;
    if (alpha == 0.0) {
        GemmConfig dummy{VAR_DIRECT, 4, 4, 1, 1};
        // alpha == 0 or k == 0 with beta == 0 writes zeros without reading
        return status(launch_dgemm(false, false, m, n, 0, 0.0, B, ldb, B, ldb, 0.0, B, ldb, batch,
                                   dummy, 0, nullptr, s));
    }
    const int sd = is_r(side) ? 1 : 0, up = is_u(uplo) ? 1 : 0, tr = is_t(ta) ? 1 : 0,
              un = is_u(diag) ? 1 : 0;
    TrsmConfig cfg = choose_trsm(sd, up, tr, un, m, n, batch);
    return status(launch_dtrsm(sd, up, tr, un, m, n, alpha, A, lda, B, ldb, batch, cfg, nullptr, s));
}

int check_potrf(char uplo, int n, const void* A, int lda, int batch, long long strideA, bool strided,
                int pos_uplo, int pos_n, int pos_A, int pos_lda, int pos_sA, int pos_batch) {
    if (!(is_l(uplo) || is_u(uplo))) return -pos_uplo;
    if (n < 0) return -pos_n;
    if (lda < imax1(n)) return -pos_lda;
    if (pos_batch && batch < 0) return -pos_batch;
    if (strided && batch > 1 && strideA < (long long)lda * n) return -pos_sA;
    if (n > 0 && batch != 0 && !A) return -pos_A;
    return 0;
}

int run_potrf(char uplo, int n, MatRef A, int lda, int* info, long long batch, cudaStream_t s) {
    PotrfConfig cfg = choose_potrf(n, lda, batch);
    return status(launch_dpotrf(n, A, lda, batch, info, cfg, s, is_u(uplo) ? 1 : 0));
}

}  // namespace

extern "C" {

int bf_dgemm(char transa, char transb, int m, int n, int k, double alpha, const double* A, int lda,
             const double* B, int ldb, double beta, double* C, int ldc, bf_stream_t stream) {
    GemmPos pos{1, 2, 3, 4, 5, 7, 8, 9, 10, 12, 13, 0, 0};
    int r = check_gemm(transa, transb, m, n, k, A, lda, B, ldb, C, ldc, 0, 1, alpha, beta, pos);
    if (r) return r;
    return run_gemm(transa, transb, m, n, k, alpha, mat_strided(A, 0), lda, mat_strided(B, 0), ldb, beta,
                    mat_strided(C, 0), ldc, 1, (cudaStream_t)stream);
}

int bf_dgemm_strided_batched(char transa, char transb, int m, int n, int k, double alpha,
                             const double* A, int lda, long long strideA, const double* B, int ldb,
                             long long strideB, double beta, double* C, int ldc, long long strideC,
                             int batch, bf_stream_t stream) {
    GemmPos pos{1, 2, 3, 4, 5, 7, 8, 10, 11, 14, 15, 16, 17};
    int r = check_gemm(transa, transb, m, n, k, A, lda, B, ldb, C, ldc, strideC, batch, alpha, beta, pos);
    if (r) return r;
    if (strideA < 0) return -9;
    if (strideB < 0) return -12;
    return run_gemm(transa, transb, m, n, k, alpha, mat_strided(A, strideA), lda, mat_strided(B, strideB),
                    ldb, beta, mat_strided(C, strideC), ldc, batch, (cudaStream_t)stream);
}

int bf_dgemm_batched(char transa, char transb, int m, int n, int k, double alpha,
                     const double* const* Aarray, int lda, const double* const* Barray, int ldb,
                     double beta, double* const* Carray, int ldc, int batch, bf_stream_t stream) {
    GemmPos pos{1, 2, 3, 4, 5, 7, 8, 9, 10, 12, 13, 0, 14};
    int r = check_gemm(transa, transb, m, n, k, Aarray, lda, Barray, ldb, Carray, ldc, 0, batch, alpha,
                       beta, pos);
    if (r) return r;
    return run_gemm(transa, transb, m, n, k, alpha, mat_array(Aarray, 0), lda, mat_array(Barray, 0), ldb,
                    beta, mat_array((const double* const*)Carray, 0), ldc, batch, (cudaStream_t)stream);
}

int bf_dtrsm(char side, char uplo, char transa, char diag, int m, int n, double alpha, const double* A,
             int lda, double* B, int ldb, bf_stream_t stream) {
    TrsmPos pos{1, 2, 3, 4, 5, 6, 8, 9, 10, 11, 0, 0};
    int r = check_trsm(side, uplo, transa, diag, m, n, A, lda, B, ldb, 0, 1, alpha, pos);
    if (r) return r;
    return run_trsm(side, uplo, transa, diag, m, n, alpha, mat_strided(A, 0), lda, mat_strided(B, 0), ldb,
                    1, (cudaStream_t)stream);
}

int bf_dtrsm_strided_batched(char side, char uplo, char transa, char diag, int m, int n, double alpha,
                             const double* A, int lda, long long strideA, double* B, int ldb,
                             long long strideB, int batch, bf_stream_t stream) {
    TrsmPos pos{1, 2, 3, 4, 5, 6, 8, 9, 11, 12, 13, 14};
    int r = check_trsm(side, uplo, transa, diag, m, n, A, lda, B, ldb, strideB, batch, alpha, pos);
    if (r) return r;
    if (strideA < 0) return -10;
    return run_trsm(side, uplo, transa, diag, m, n, alpha, mat_strided(A, strideA), lda,
                    mat_strided(B, strideB), ldb, batch, (cudaStream_t)stream);
}

int bf_dtrsm_batched(char side, char uplo, char transa, char diag, int m, int n, double alpha,
                     const double* const* Aarray, int lda, double* const* Barray, int ldb, int batch,
                     bf_stream_t stream) {
    TrsmPos pos{1, 2, 3, 4, 5, 6, 8, 9, 10, 11, 0, 12};
    int r = check_trsm(side, uplo, transa, diag, m, n, Aarray, lda, Barray, ldb, 0, batch, alpha, pos);
    if (r) return r;
    return run_trsm(side, uplo, transa, diag, m, n, alpha, mat_array(Aarray, 0), lda,
                    mat_array((const double* const*)Barray, 0), ldb, batch, (cudaStream_t)stream);
}

int bf_dpotrf(char uplo, int n, double* A, int lda, int* info, bf_stream_t stream) {
    int r = check_potrf(uplo, n, A, lda, 1, 0, false, 1, 2, 3, 4, 0, 0);
    if (r) return r;
    return run_potrf(uplo, n, mat_strided(A, 0), lda, info, 1, (cudaStream_t)stream);
}

int bf_dpotrf_strided_batched(char uplo, int n, double* A, int lda, long long strideA, int* info,
                              int batch, bf_stream_t stream) {
    int r = check_potrf(uplo, n, A, lda, batch, strideA, true, 1, 2, 3, 4, 5, 7);
    if (r) return r;
    return run_potrf(uplo, n, mat_strided(A, strideA), lda, info, batch, (cudaStream_t)stream);
}

int bf_dpotrf_batched(char uplo, int n, double* const* Aarray, int lda, int* info, int batch,
                      bf_stream_t stream) {
    int r = check_potrf(uplo, n, Aarray, lda, batch, 0, false, 1, 2, 3, 4, 0, 6);
    if (r) return r;
    return run_potrf(uplo, n, mat_array((const double* const*)Aarray, 0), lda, info, batch, (cudaStream_t)stream);
}

static int potrs_run(char uplo, int n, int nrhs, MatRef A, const void* Ap, int lda, MatRef B, const void* Bp, int ldb,
                     long long strideB, int batch, bf_stream_t stream, const int* pos) {
    // pos: uplo, n, nrhs, A, lda, B, ldb, strideB, batch
    if (!(is_l(uplo) || is_u(uplo))) return -pos[0];
    if (n < 0) return -pos[1];
    if (nrhs < 0) return -pos[2];
    if (lda < imax1(n)) return -pos[4];
    if (ldb < imax1(n)) return -pos[6];
    if (pos[8] && batch < 0) return -pos[8];
    if (pos[7] && batch > 1 && strideB < (long long)ldb * nrhs) return -pos[7];
    const bool work = n > 0 && nrhs > 0 && batch > 0;
    if (work && !Ap) return -pos[3];
    if (work && !Bp) return -pos[5];
    if (!work) return 0;
    // 'L': L Y = B, L^T X = Y;  'U': U^T Y = B, U X = Y
    const char u = is_u(uplo) ? 'U' : 'L';
    int r = run_trsm('L', u, u == 'L' ? 'N' : 'T', 'N', n, nrhs, 1.0, A, lda, B, ldb, batch, (cudaStream_t)stream);
    if (r) return r;
    return run_trsm('L', u, u == 'L' ? 'T' : 'N', 'N', n, nrhs, 1.0, A, lda, B, ldb, batch, (cudaStream_t)stream);
}

static int potrs_impl(char uplo, int n, int nrhs, const double* A, int lda, long long strideA, double* B,
                      int ldb, long long strideB, int batch, bf_stream_t stream, const int* pos) {
    return potrs_run(uplo, n, nrhs, mat_strided(A, strideA), A, lda, mat_strided(B, strideB), B, ldb, strideB, batch,
                     stream, pos);
}

int bf_dpotrs(char uplo, int n, int nrhs, const double* A, int lda, double* B, int ldb, bf_stream_t stream) {
    static const int pos[9] = {1, 2, 3, 4, 5, 6, 7, 0, 0};
    return potrs_impl(uplo, n, nrhs, A, lda, 0, B, ldb, 0, 1, stream, pos);
}

int bf_dpotrs_strided_batched(char uplo, int n, int nrhs, const double* A, int lda, long long strideA,
                              double* B, int ldb, long long strideB, int batch, bf_stream_t stream) {
    static const int pos[9] = {1, 2, 3, 4, 5, 7, 8, 9, 10};
    if (strideA < 0) return -6;
    return potrs_impl(uplo, n, nrhs, A, lda, strideA, B, ldb, strideB, batch, stream, pos);
}

int bf_dpotrs_batched(char uplo, int n, int nrhs, const double* const* Aarray, int lda, double* const* Barray,
                      int ldb, int batch, bf_stream_t stream) {
    static const int pos[9] = {1, 2, 3, 4, 5, 6, 7, 0, 8};
    return potrs_run(uplo, n, nrhs, mat_array(Aarray, 0), Aarray, lda, mat_array((const double* const*)Barray, 0),
                     Barray, ldb, 0, batch, stream, pos);
}

// ------------------------------------------------------------------------ dsyrk
static int syrk_impl(char uplo, char trans, int n, int k, double alpha, MatRef A, const void* Ap, int lda,
                     double beta, MatRef C, const void* Cp, int ldc, long long strideC, int batch, bool strided,
                     bf_stream_t stream, const int* pos) {
    // pos: uplo, trans, n, k, A, lda, C, ldc, strideC, batch
    if (!(is_l(uplo) || is_u(uplo))) return -pos[0];
    if (!(is_n(trans) || is_t(trans))) return -pos[1];
    if (n < 0) return -pos[2];
    if (k < 0) return -pos[3];
    if (lda < imax1(is_n(trans) ? n : k)) return -pos[5];
    if (ldc < imax1(n)) return -pos[7];
    if (pos[9] && batch < 0) return -pos[9];
    if (strided && batch > 1 && strideC < (long long)ldc * n) return -pos[8];
    const bool work = n > 0 && batch > 0;
    if (work && k > 0 && alpha != 0.0 && !Ap) return -pos[4];
    if (work && !Cp) return -pos[6];
    if (!work) return 0;
    return status(launch_dsyrk(is_u(uplo) ? 1 : 0, is_t(trans) ? 1 : 0, n, k, alpha, A, lda, beta, C, ldc, batch,
                               (cudaStream_t)stream));
}

int bf_dsyrk(char uplo, char trans, int n, int k, double alpha, const double* A, int lda, double beta, double* C,
             int ldc, bf_stream_t stream) {
    static const int pos[10] = {1, 2, 3, 4, 6, 7, 9, 10, 0, 0};
    return syrk_impl(uplo, trans, n, k, alpha, mat_strided(A, 0), A, lda, beta, mat_strided(C, 0), C, ldc, 0, 1,
                     false, stream, pos);
}

int bf_dsyrk_strided_batched(char uplo, char trans, int n, int k, double alpha, const double* A, int lda,
                             long long strideA, double beta, double* C, int ldc, long long strideC, int batch,
                             bf_stream_t stream) {
    static const int pos[10] = {1, 2, 3, 4, 6, 7, 10, 11, 12, 13};
    if (strideA < 0) return -8;
    return syrk_impl(uplo, trans, n, k, alpha, mat_strided(A, strideA), A, lda, beta, mat_strided(C, strideC), C,
                     ldc, strideC, batch, true, stream, pos);
}

int bf_dsyrk_batched(char uplo, char trans, int n, int k, double alpha, const double* const* Aarray, int lda,
                     double beta, double* const* Carray, int ldc, int batch, bf_stream_t stream) {
    static const int pos[10] = {1, 2, 3, 4, 6, 7, 9, 10, 0, 11};
    return syrk_impl(uplo, trans, n, k, alpha, mat_array(Aarray, 0), Aarray, lda, beta,
                     mat_array((const double* const*)Carray, 0), Carray, ldc, 0, batch, false, stream, pos);
}

// ------------------------------------------------------------------------ dsyrk + dpotrf
static int syrk_potrf_impl(int n, int k, MatRef A, const void* Ap, int lda, MatRef C, const void* Cp, int ldc,
                           long long strideC, int* info, int batch, bool strided, bf_stream_t stream,
                           const int* pos) {
    // pos: n, k, A, lda, C, ldc, strideC, batch
    if (n < 0) return -pos[0];
    if (k < 0) return -pos[1];
    if (lda < imax1(n)) return -pos[3];
    if (ldc < imax1(n)) return -pos[5];
    if (pos[7] && batch < 0) return -pos[7];
    if (strided && batch > 1 && strideC < (long long)ldc * n) return -pos[6];
    const bool work = n > 0 && batch > 0;
    if (work && k > 0 && !Ap) return -pos[2];
    if (work && !Cp) return -pos[4];
    if (batch <= 0) return 0;
    return status(launch_dsyrk_dpotrf(n, k, A, lda, C, ldc, batch, info, (cudaStream_t)stream));
}

int bf_dsyrk_dpotrf(int n, int k, const double* A, int lda, double* C, int ldc, int* info, bf_stream_t stream) {
    static const int pos[8] = {1, 2, 3, 4, 5, 6, 0, 0};
    return syrk_potrf_impl(n, k, mat_strided(A, 0), A, lda, mat_strided(C, 0), C, ldc, 0, info, 1, false, stream,
                           pos);
}

int bf_dsyrk_dpotrf_strided_batched(int n, int k, const double* A, int lda, long long strideA, double* C, int ldc,
                                    long long strideC, int* info, int batch, bf_stream_t stream) {
    static const int pos[8] = {1, 2, 3, 4, 6, 7, 8, 10};
    if (strideA < 0) return -5;
    return syrk_potrf_impl(n, k, mat_strided(A, strideA), A, lda, mat_strided(C, strideC), C, ldc, strideC, info,
                           batch, true, stream, pos);
}

// ------------------------------------------------------------------------ dtrmm
static int trmm_impl(char side, char uplo, char ta, char diag, int m, int n, double alpha, MatRef A, const void* Ap,
                     int lda, MatRef B, const void* Bp, int ldb, long long strideB, int batch, bool strided,
                     bf_stream_t stream, const int* pos) {
    // pos: side, uplo, ta, diag, m, n, A, lda, B, ldb, strideB, batch
    if (!(is_l(side) || is_r(side))) return -pos[0];
    if (!(is_l(uplo) || is_u(uplo))) return -pos[1];
    if (!(is_n(ta) || is_t(ta))) return -pos[2];
    if (!(is_u(diag) || is_n(diag))) return -pos[3];
    if (m < 0) return -pos[4];
    if (n < 0) return -pos[5];
    if (lda < imax1(is_l(side) ? m : n)) return -pos[7];
    if (ldb < imax1(m)) return -pos[9];
    if (pos[11] && batch < 0) return -pos[11];
    if (strided && batch > 1 && strideB < (long long)ldb * n) return -pos[10];
    const bool work = m > 0 && n > 0 && batch > 0;
    if (work && alpha != 0.0 && !Ap) return -pos[6];
    if (work && !Bp) return -pos[8];
    if (!work) return 0;
    if (alpha == 0.0) {  // B <= 0 without reading A or B
        GemmConfig dummy{VAR_DIRECT, 4, 4, 1, 1};
        return status(launch_dgemm(false, false, m, n, 0, 0.0, B, ldb, B, ldb, 0.0, B, ldb, batch, dummy, 0, nullptr,
                                   (cudaStream_t)stream));
    }
    const int right = is_r(side) ? 1 : 0;
    const int rows = right ? m : n;  // independent rows of the right-side form
    return status(launch_dtrmm(right, is_u(uplo) ? 1 : 0, is_t(ta) ? 1 : 0, is_u(diag) ? 1 : 0, m, n, alpha, A, lda,
                               B, ldb, batch, rows >= 256 ? 8 : 4, (cudaStream_t)stream));
}

int bf_dtrmm(char side, char uplo, char transa, char diag, int m, int n, double alpha, const double* A, int lda,
             double* B, int ldb, bf_stream_t stream) {
    static const int pos[12] = {1, 2, 3, 4, 5, 6, 8, 9, 10, 11, 0, 0};
    return trmm_impl(side, uplo, transa, diag, m, n, alpha, mat_strided(A, 0), A, lda, mat_strided(B, 0), B, ldb, 0,
                     1, false, stream, pos);
}

int bf_dtrmm_strided_batched(char side, char uplo, char transa, char diag, int m, int n, double alpha,
                             const double* A, int lda, long long strideA, double* B, int ldb, long long strideB,
                             int batch, bf_stream_t stream) {
    static const int pos[12] = {1, 2, 3, 4, 5, 6, 8, 9, 11, 12, 13, 14};
    if (strideA < 0) return -10;
    return trmm_impl(side, uplo, transa, diag, m, n, alpha, mat_strided(A, strideA), A, lda, mat_strided(B, strideB),
                     B, ldb, strideB, batch, true, stream, pos);
}

int bf_dtrmm_batched(char side, char uplo, char transa, char diag, int m, int n, double alpha,
                     const double* const* Aarray, int lda, double* const* Barray, int ldb, int batch,
                     bf_stream_t stream) {
    static const int pos[12] = {1, 2, 3, 4, 5, 6, 8, 9, 10, 11, 0, 12};
    return trmm_impl(side, uplo, transa, diag, m, n, alpha, mat_array(Aarray, 0), Aarray, lda,
                     mat_array((const double* const*)Barray, 0), Barray, ldb, 0, batch, false, stream, pos);
}

// ------------------------------------------------------------------------ dgetrf / dgetrs
static int getrf_impl(int m, int n, double* A, int lda, long long strideA, int* ipiv, long long strideIpiv,
                      int* info, int batch, bool strided, bf_stream_t stream, const int* pos) {
    // pos: m, n, A, lda, strideA, ipiv, strideIpiv, batch
    if (m < 0) return -pos[0];
    if (n < 0) return -pos[1];
    if (lda < imax1(m)) return -pos[3];
    if (pos[7] && batch < 0) return -pos[7];
    if (strided && batch > 1 && strideA < (long long)lda * n) return -pos[4];
    const int mn = m < n ? m : n;
    if (strided && batch > 1 && strideIpiv < mn) return -pos[6];
    const bool work = mn > 0 && batch > 0;
    if (work && !A) return -pos[2];
    if (work && !ipiv) return -pos[5];
    if (m != n && m > kGetrfMaxRows) return BF_ERR_NOT_SUPPORTED;
    if (batch <= 0) return 0;
    return status(launch_dgetrf(m, n, mat_strided(A, strideA), lda, ipiv, strided ? strideIpiv : mn, info, batch,
                                (cudaStream_t)stream));
}

int bf_dgetrf(int m, int n, double* A, int lda, int* ipiv, int* info, bf_stream_t stream) {
    static const int pos[8] = {1, 2, 3, 4, 0, 5, 0, 0};
    return getrf_impl(m, n, A, lda, 0, ipiv, 0, info, 1, false, stream, pos);
}

int bf_dgetrf_strided_batched(int m, int n, double* A, int lda, long long strideA, int* ipiv, long long strideIpiv,
                              int* info, int batch, bf_stream_t stream) {
    static const int pos[8] = {1, 2, 3, 4, 5, 6, 7, 9};
    if (strideA < 0) return -5;
    return getrf_impl(m, n, A, lda, strideA, ipiv, strideIpiv, info, batch, true, stream, pos);
}

static int getrs_impl(char trans, int n, int nrhs, const double* A, int lda, long long strideA, const int* ipiv,
                      long long strideIpiv, double* B, int ldb, long long strideB, int batch, bool strided,
                      bf_stream_t stream, const int* pos) {
    // pos: trans, n, nrhs, A, lda, ipiv, B, ldb, strideB, batch
    if (!(is_n(trans) || is_t(trans))) return -pos[0];
    if (n < 0) return -pos[1];
    if (nrhs < 0) return -pos[2];
    if (lda < imax1(n)) return -pos[4];
    if (ldb < imax1(n)) return -pos[7];
    if (pos[9] && batch < 0) return -pos[9];
    if (strided && batch > 1 && strideB < (long long)ldb * nrhs) return -pos[8];
    const bool work = n > 0 && nrhs > 0 && batch > 0;
    if (work && !A) return -pos[3];
    if (work && !ipiv) return -pos[5];
    if (work && !B) return -pos[6];
    if (!work) return 0;
    return status(launch_dgetrs(is_t(trans) ? 1 : 0, n, nrhs, mat_strided(A, strideA), lda, ipiv,
                                strided ? strideIpiv : n, mat_strided(B, strideB), ldb, batch, (cudaStream_t)stream));
}

int bf_dgetrs(char trans, int n, int nrhs, const double* A, int lda, const int* ipiv, double* B, int ldb,
              bf_stream_t stream) {
    static const int pos[10] = {1, 2, 3, 4, 5, 6, 7, 8, 0, 0};
    return getrs_impl(trans, n, nrhs, A, lda, 0, ipiv, 0, B, ldb, 0, 1, false, stream, pos);
}

int bf_dgetrs_strided_batched(char trans, int n, int nrhs, const double* A, int lda, long long strideA,
                              const int* ipiv, long long strideIpiv, double* B, int ldb, long long strideB, int batch,
                              bf_stream_t stream) {
    static const int pos[10] = {1, 2, 3, 4, 5, 7, 9, 10, 11, 12};
    if (strideA < 0) return -6;
    if (batch > 1 && strideIpiv < n) return -8;
    return getrs_impl(trans, n, nrhs, A, lda, strideA, ipiv, strideIpiv, B, ldb, strideB, batch, true, stream, pos);
}

const char* bf_status_string(int s) {
    if (s == BF_SUCCESS) return "success";
    if (s == BF_ERR_CUDA) return "a CUDA launch failed";
    if (s == BF_ERR_NOT_SUPPORTED) return "option not supported by this library";
    if (s == BF_ERR_NOALLOC_LIMIT)
        return "problem count exceeds the allocation-free scratch limit (BF_RAGGED_NOALLOC_MAX)";
    if (s < 0) return "illegal argument (the value is minus its 1-based position)";
    return "unknown status";
}

}  // extern "C"
