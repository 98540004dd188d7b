// bf_tiny.cu -- dgemm (m, n, k <= 4) and dtrsm (orders <= 8) for tiny problems: one thread
// per whole problem, the CTA's problems staged through shared memory (bf_stage.cuh).
//
// At these sizes a problem is a few hundred bytes and a few dozen fused multiply-adds, so the
// kernels sit at the ridge of the roofline.  The direct kernels read every problem through
// L1 with one problem per few lanes: each warp load touches 32 separate cache lines.  Here the
// CTA reads its problems as one run of 16-byte coalesced pieces (the packed variants of
// section 2.2, with the buffer in shared memory), every thread computes its problem from a
// bank-staggered, problem-interleaved copy, and the results go back the same way.
#include "bf_internal.h"
#include "bf_stage.cuh"

namespace bf {

template <bool TA, bool TB, bool NEG>
__global__ void __launch_bounds__(128) dgemm_tiny_kernel(GemmParams p) {
    extern __shared__ double smem[];
    const int T = blockDim.x, ST = T + 1;
    const long long q0 = blockIdx.x * (long long)T;
    const int nq = (int)((p.batch - q0) < T ? (p.batch - q0) : T);
    const int m = p.m, n = p.n, k = p.k;
    const int ra = TA ? k : m, ca = TA ? m : k, rb = TB ? n : k, cb = TB ? k : n;
    double* sA = smem;
    double* sB = sA + ra * ca * ST;
    double* sC = sB + rb * cb * ST;
    const bool readC = p.mode == ACC_C || p.mode == ACC_BC || (p.mode == ACC_GEN && p.beta != 0.0) || p.skip;
    stage_in(p.A, ra, ca, p.lda, false, q0, nq, sA, ST);
    stage_in(p.B, rb, cb, p.ldb, false, q0, nq, sB, ST);
    if (readC) stage_in(p.C, m, n, p.ldc, false, q0, nq, sC, ST);
    stage_wait();
    __syncthreads();
    const int t = threadIdx.x;
    if (t < nq && !(p.skip && p.skip[q0 + t] != 0)) {
        double a[4][4], b[4][4], acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int pp = 0; pp < 4; pp++)
                a[i][pp] = (i < m && pp < k) ? (TA ? sA[(pp + i * ra) * ST + t] : sA[(i + pp * ra) * ST + t]) : 0.0;
#pragma unroll
        for (int pp = 0; pp < 4; pp++)
#pragma unroll
            for (int j = 0; j < 4; j++)
                b[pp][j] = (pp < k && j < n) ? (TB ? sB[(j + pp * rb) * ST + t] : sB[(pp + j * rb) * ST + t]) : 0.0;
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) {
                double c0 = 0.0;
                if ((p.mode == ACC_C || p.mode == ACC_BC) && i < m && j < n) c0 = sC[(i + j * m) * ST + t];
                acc[i][j] = (p.mode == ACC_BC) ? p.beta * c0 : c0;
            }
#pragma unroll
        for (int pp = 0; pp < 4; pp++)
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++)
                    acc[i][j] = NEG ? fma(-a[i][pp], b[pp][j], acc[i][j]) : fma(a[i][pp], b[pp][j], acc[i][j]);
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (i < m && j < n) {
                    double* cp = sC + (i + j * m) * ST + t;
                    double v = acc[i][j];
                    if (p.mode == ACC_GEN) v = (p.beta == 0.0) ? p.alpha * v : fma(p.alpha, v, p.beta * *cp);
                    *cp = v;
                }
            }
    }
    __syncthreads();
    stage_out(p.C, m, n, p.ldc, false, q0, nq, sC, ST, true, [](int, int) { return true; });
}

size_t tiny_gemm_smem(int m, int n, int k, int T) {
    return sizeof(double) * (size_t)(T + 1) * ((size_t)m * k + (size_t)k * n + (size_t)m * n);
}

template <class K>
static cudaError_t allow_smem(K kfn, size_t smem) {
    if (smem + kStaticSmemSlack <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_dgemm_tiny(bool ta, bool tb, bool neg, const GemmParams& p, cudaStream_t s) {
    const int T = 128;
    const size_t smem = tiny_gemm_smem(p.m, p.n, p.k, T);
    const unsigned blocks = (unsigned)((p.batch + T - 1) / T);
    cudaError_t e;
#define BF_TINY_CASE(A_, B_)                                                                          \
    if (ta == A_ && tb == B_) {                                                                       \
        if (neg) {                                                                                    \
            if ((e = allow_smem(dgemm_tiny_kernel<A_, B_, true>, smem)) != cudaSuccess) return e;     \
            dgemm_tiny_kernel<A_, B_, true><<<blocks, T, smem, s>>>(p);                               \
        } else {                                                                                      \
            if ((e = allow_smem(dgemm_tiny_kernel<A_, B_, false>, smem)) != cudaSuccess) return e;    \
            dgemm_tiny_kernel<A_, B_, false><<<blocks, T, smem, s>>>(p);                              \
        }                                                                                             \
    }
    BF_TINY_CASE(false, false)
    BF_TINY_CASE(false, true)
    BF_TINY_CASE(true, false)
    BF_TINY_CASE(true, true)
#undef BF_TINY_CASE
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ dtrsm, orders <= 8
// op(A) X = alpha B (left, A m x m) or X op(A) = alpha B (right, A n x n); B m x n.
template <bool RIGHT>
__global__ void __launch_bounds__(128) dtrsm_tiny_kernel(TrsmParams p) {
    extern __shared__ double smem[];
    const int T = blockDim.x, ST = T + 1;
    const long long q0 = blockIdx.x * (long long)T;
    const int nq = (int)((p.batch - q0) < T ? (p.batch - q0) : T);
    const int m = p.m, n = p.n;         // B is m x n
    const int ka = RIGHT ? n : m;       // order of A
    double* sA = smem;
    double* sB = sA + ka * ka * ST;
    stage_in(p.A, ka, ka, p.lda, false, q0, nq, sA, ST);
    stage_in(p.B, m, n, p.ldb, false, q0, nq, sB, ST);
    stage_wait();
    __syncthreads();
    const int t = threadIdx.x;
    if (t < nq && !(p.skip && p.skip[q0 + t] != 0)) {
        // T(i, j) = op(A)(i, j); lower when (stored lower, no transpose) or (stored upper, transpose)
        auto Tel = [&](int i, int j) -> double {
            return p.et ? sA[(j + i * ka) * ST + t] : sA[(i + j * ka) * ST + t];
        };
        const bool lower = p.upper == 0;
        double rinv[8];
#pragma unroll
        for (int j = 0; j < 8; j++) rinv[j] = (j < ka && !p.unit) ? 1.0 / Tel(j, j) : 1.0;
        if (RIGHT) {
            // every row r: x T = alpha b; T lower -> columns from n-1 down, upper -> from 0 up
            for (int r = 0; r < m; r++) {
                double x[8];
#pragma unroll
                for (int j = 0; j < 8; j++) x[j] = (j < n) ? p.alpha * sB[(r + j * m) * ST + t] : 0.0;
#pragma unroll
                for (int jj = 0; jj < 8; jj++) {
                    const int j = lower ? 7 - jj : jj;
                    if (j < n) {
                        double sacc = x[j];
#pragma unroll
                        for (int pp = 0; pp < 8; pp++) {
                            const bool after = lower ? (pp > j) : (pp < j);
                            if (after && pp < n) sacc = fma(-x[pp], Tel(pp, j), sacc);
                        }
                        x[j] = sacc * rinv[j];
                    }
                }
#pragma unroll
                for (int j = 0; j < 8; j++)
                    if (j < n) sB[(r + j * m) * ST + t] = x[j];
            }
        } else {
            // every column c: T x = alpha b; T lower -> rows from 0 up, upper -> from m-1 down
            for (int c = 0; c < n; c++) {
                double x[8];
#pragma unroll
                for (int i = 0; i < 8; i++) x[i] = (i < m) ? p.alpha * sB[(i + c * m) * ST + t] : 0.0;
#pragma unroll
                for (int ii = 0; ii < 8; ii++) {
                    const int i = lower ? ii : 7 - ii;
                    if (i < m) {
                        double sacc = x[i];
#pragma unroll
                        for (int pp = 0; pp < 8; pp++) {
                            const bool before = lower ? (pp < i) : (pp > i);
                            if (before && pp < m) sacc = fma(-Tel(i, pp), x[pp], sacc);
                        }
                        x[i] = sacc * rinv[i];
                    }
                }
#pragma unroll
                for (int i = 0; i < 8; i++)
                    if (i < m) sB[(i + c * m) * ST + t] = x[i];
            }
        }
    }
    __syncthreads();
    stage_out(p.B, m, n, p.ldb, false, q0, nq, sB, ST, true, [](int, int) { return true; });
}

cudaError_t launch_dtrsm_tiny(int side, int uplo, int trans, int unit, int m, int n, double alpha, MatRef A, int lda,
                              MatRef B, int ldb, long long batch, const int* skip, cudaStream_t s) {
    TrsmParams p;
    p.m = m; p.n = n; p.alpha = alpha;
    p.A = A; p.lda = lda; p.B = B; p.ldb = ldb; p.batch = batch;
    p.bt = 0;
    p.et = trans;
    p.upper = ((uplo == 1) ^ trans) ? 1 : 0;  // op(A) upper
    p.unit = unit;
    p.tpp = 1; p.P = 1;
    p.skip = skip;
    const int ka = side == 1 ? n : m;
    const size_t per = (size_t)ka * ka + (size_t)m * n;
    const int T = sizeof(double) * 129 * per <= 64 * 1024 ? 128 : 64;
    const size_t smem = sizeof(double) * (size_t)(T + 1) * per;
    const unsigned blocks = (unsigned)((batch + T - 1) / T);
    cudaError_t e;
    if (side == 1) {
        if ((e = allow_smem(dtrsm_tiny_kernel<true>, smem)) != cudaSuccess) return e;
        dtrsm_tiny_kernel<true><<<blocks, T, smem, s>>>(p);
    } else {
        if ((e = allow_smem(dtrsm_tiny_kernel<false>, smem)) != cudaSuccess) return e;
        dtrsm_tiny_kernel<false><<<blocks, T, smem, s>>>(p);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace bf
