// bf_dsposv.cu -- batched mixed-precision SPD solve: binary32 Cholesky factor,
// binary64 iterative refinement (the interface is LAPACK's dsposv).
//
// The factorisation and solves are the paper's dpotrf/dtrsm (section 3.1)
// carried out in binary32; refinement recovers binary64 accuracy:
//   1. A (binary64, lower triangle referenced) is rounded to binary32 into
//      shared memory and factored A32 = L32 L32^T, right-looking with 8-column
//      panels.  Each pivot is tested for positivity and square-rooted in
//      binary64, then rounded to binary32.
//   2. x = L32^{-T} L32^{-1} b (binary32 substitutions, x kept in binary64).
//   3. repeat: r = b - A x in binary64 (A read from global memory, symmetric
//      from its lower triangle); stop when the normwise backward error
//      eta = ||r||_inf / (||A||_inf ||x||_inf + ||b||_inf) <= tol;
//      d = L32^{-T} L32^{-1} r (binary32); x = x + d in binary64.
//   4. If the binary32 factorisation fails or `itmax` refinement steps do not
//      reach tol, the problem is factored and solved in binary64 instead and
//      iter = -1 (LAPACK's dsposv rule).
// ||A||_inf is accumulated in binary32 from the rounded matrix and scaled by
// (1 - 2(n+1) 2^-24), a lower bound of the binary64 norm, so the stopping
// test never under-estimates eta.
//
// One CTA (256 threads) per problem; n <= BF_DSPOSV_NMAX.
#include "bf_internal.h"
#include "../../include/bfgpu.h"

namespace bf {

struct SposvParams {
    int n, nrhs;
    MatRef A;
    int lda;
    MatRef B;
    int ldb;
    MatRef X;
    int ldx;
    int* iter;
    int* info;
    double tol;
    int itmax;
    long long batch;
};

static __host__ __device__ inline size_t sposv_mat_bytes(int n) {
    size_t f32 = (size_t)n * (n + 1) * sizeof(float);
    size_t f64 = (size_t)n * (n + 1) / 2 * sizeof(double);
    size_t m = f32 > f64 ? f32 : f64;
    return (m + 15) / 16 * 16;
}

static size_t sposv_smem_bytes(int n) {
    // matrix | x, r (binary64) | w, rinv (binary32) | reduction scratch
    return sposv_mat_bytes(n) + 2 * (size_t)n * sizeof(double) + 2 * (size_t)((n + 3) / 4 * 4) * sizeof(float) +
           64 * sizeof(double);
}

// |v| of a non-negative or NaN-free double as an order-preserving integer
__device__ __forceinline__ unsigned long long absbits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// block-wide max of non-negative doubles (as bit patterns); all threads get the result
__device__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* scratch) {
    v = warp_max_u64(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) scratch[w] = v;
    __syncthreads();
    unsigned long long r = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) r = scratch[i] > r ? scratch[i] : r;
    return r;
}

// binary32 substitutions with the factor in shared memory, one warp:
// w <- L^{-T} L^{-1} w  (rinv holds 1 / l_jj)
__device__ void solve32_warp(const float* L, int ld, const float* rinv, float* w, int n) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < n; j++) {
        const float wj = w[j] * rinv[j];
        __syncwarp();
        if (lane == 0) w[j] = wj;
        for (int i = j + 1 + lane; i < n; i += 32) w[i] = fmaf(-L[i + j * ld], wj, w[i]);
        __syncwarp();
    }
    for (int j = n - 1; j >= 0; j--) {
        const float wj = w[j] * rinv[j];
        __syncwarp();
        if (lane == 0) w[j] = wj;
        for (int i = lane; i < j; i += 32) w[i] = fmaf(-L[j + i * ld], wj, w[i]);
        __syncwarp();
    }
}

// packed lower index (column-major)
__device__ __forceinline__ int pk(int i, int j, int n) { return j * n - (j * (j - 1)) / 2 + (i - j); }

__global__ void __launch_bounds__(256) dsposv_kernel(SposvParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const long long q = blockIdx.x;
    if (q >= p.batch) return;
    const int n = p.n;
    const int tid = threadIdx.x, T = blockDim.x, warp = tid >> 5, lane = tid & 31;
    const int ld = n + 1;
    float* L = reinterpret_cast<float*>(smem_raw);
    double* Lp = reinterpret_cast<double*>(smem_raw);  // binary64 fallback (packed lower)
    double* xv = reinterpret_cast<double*>(smem_raw + sposv_mat_bytes(n));
    double* rv = xv + n;
    float* wv = reinterpret_cast<float*>(rv + n);
    float* rinv = wv + (n + 3) / 4 * 4;
    unsigned long long* scratch = reinterpret_cast<unsigned long long*>(rinv + (n + 3) / 4 * 4);
    __shared__ int s_flag;
    __shared__ double s_anorm;

    const double* A = p.A.ptr(q);
    const double* B = p.B.ptr(q);
    double* X = p.X.mptr(q);

    // ---- 1. round the lower triangle to binary32 ----
    for (int e = tid; e < n * n; e += T) {
        const int j = e / n, i = e - j * n;
        if (i >= j) L[i + j * ld] = (float)A[i + (long long)j * p.lda];
    }
    __syncthreads();
    // ||A||_inf of the symmetric matrix, binary32 sums of the rounded entries
    unsigned long long an = 0;
    for (int i = tid; i < n; i += T) {
        float s = 0.0f;
        for (int j = 0; j < n; j++) s += fabsf(j <= i ? L[i + j * ld] : L[j + i * ld]);
        an = (unsigned long long)__double_as_longlong((double)s) > an ? (unsigned long long)__double_as_longlong((double)s) : an;
    }
    an = block_max_u64(an, scratch);
    if (tid == 0) s_anorm = __longlong_as_double((long long)an) * (1.0 - 2.0 * (n + 1) * 5.9604644775390625e-08);

    // ---- 2. binary32 Cholesky, right-looking, 8-column panels ----
    if (tid == 0) s_flag = 0;
    __syncthreads();
    for (int J = 0; J < n; J += 8) {
        const int nb = imin(8, n - J);
        if (warp == 0) {
            for (int c = 0; c < nb; c++) {
                const int j = J + c;
                const double d = (double)L[j + j * ld];
                if (!(d > 0.0)) {  // every lane sees the same value
                    if (lane == 0) s_flag = j + 1;
                    break;
                }
                const float ljj = (float)sqrt(d);  // pivot square root in binary64
                const float ri = 1.0f / ljj;
                __syncwarp();
                if (lane == 0) {
                    L[j + j * ld] = ljj;
                    rinv[j] = ri;
                }
                for (int i = j + 1 + lane; i < n; i += 32) L[i + j * ld] *= ri;
                __syncwarp();
                // rank-1 update of the rest of the panel
                for (int k = j + 1; k < J + nb; k++) {
                    const float lkj = L[k + j * ld];
                    for (int i = k + lane; i < n; i += 32) L[i + k * ld] = fmaf(-L[i + j * ld], lkj, L[i + k * ld]);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (s_flag) break;
        // trailing update: L22 -= L21 L21^T on lower 4x4 tiles, rank nb
        const int R = J + nb;
        const int m = n - R;
        if (m > 0) {
            const int tb = (m + 3) / 4;
            const int ntile = tb * (tb + 1) / 2;
            for (int t = tid; t < ntile; t += T) {
                // tile (I, K), I >= K, enumerated row by row of the lower tile triangle
                int I = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
                while ((I + 1) * (I + 2) / 2 <= t) I++;
                while (I * (I + 1) / 2 > t) I--;
                const int K = t - I * (I + 1) / 2;
                const int i0 = R + 4 * I, k0 = R + 4 * K;
                float acc[4][4];
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int b = 0; b < 4; b++) acc[a][b] = 0.0f;
                for (int c = 0; c < nb; c++) {
                    float li[4], lk[4];
#pragma unroll
                    for (int a = 0; a < 4; a++) li[a] = L[imin(i0 + a, n - 1) + (J + c) * ld];
#pragma unroll
                    for (int b = 0; b < 4; b++) lk[b] = L[imin(k0 + b, n - 1) + (J + c) * ld];
#pragma unroll
                    for (int a = 0; a < 4; a++)
#pragma unroll
                        for (int b = 0; b < 4; b++) acc[a][b] = fmaf(li[a], lk[b], acc[a][b]);
                }
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int b = 0; b < 4; b++) {
                        const int i = i0 + a, k = k0 + b;
                        if (i < n && k <= i) L[i + k * ld] -= acc[a][b];
                    }
            }
        }
        __syncthreads();
    }
    bool fallback = s_flag != 0;

    // ---- 3. solve and refine every right-hand side ----
    int iters = 0;
    for (int c = 0; c < p.nrhs && !fallback; c++) {
        const double* b = B + (long long)c * p.ldb;
        unsigned long long bn = 0;
        for (int i = tid; i < n; i += T) {
            const double bi = b[i];
            bn = absbits(bi) > bn ? absbits(bi) : bn;
            wv[i] = (float)bi;
        }
        bn = block_max_u64(bn, scratch);
        const double bnorm = __longlong_as_double((long long)bn);
        if (warp == 0) solve32_warp(L, ld, rinv, wv, n);
        __syncthreads();
        for (int i = tid; i < n; i += T) xv[i] = (double)wv[i];
        __syncthreads();
        int it = 0;
        bool done = false;
        for (;;) {
            // r = b - A x, binary64, A symmetric from its lower triangle
            unsigned long long rn = 0, xn = 0;
            for (int i = tid; i < n; i += T) {
                double s = b[i];
                for (int j = 0; j < n; j++) {
                    const double a = (j <= i) ? A[i + (long long)j * p.lda] : A[j + (long long)i * p.lda];
                    s = fma(-a, xv[j], s);
                }
                rv[i] = s;
                rn = absbits(s) > rn ? absbits(s) : rn;
                xn = absbits(xv[i]) > xn ? absbits(xv[i]) : xn;
            }
            rn = block_max_u64(rn, scratch);
            __syncthreads();
            xn = block_max_u64(xn, scratch);
            const double rnorm = __longlong_as_double((long long)rn);
            const double xnorm = __longlong_as_double((long long)xn);
            const double den = s_anorm * xnorm + bnorm;
            if (rnorm <= p.tol * den) {
                done = true;
                break;
            }
            if (it == p.itmax) break;
            for (int i = tid; i < n; i += T) wv[i] = (float)rv[i];
            __syncthreads();
            if (warp == 0) solve32_warp(L, ld, rinv, wv, n);
            __syncthreads();
            for (int i = tid; i < n; i += T) xv[i] += (double)wv[i];
            __syncthreads();
            it++;
        }
        if (!done) {
            fallback = true;
            break;
        }
        iters = it > iters ? it : iters;
        double* x = X + (long long)c * p.ldx;
        for (int i = tid; i < n; i += T) x[i] = xv[i];
        __syncthreads();
    }
    if (!fallback) {
        if (tid == 0) {
            if (p.iter) p.iter[q] = iters;
            if (p.info) p.info[q] = 0;
        }
        return;
    }

    // ---- 4. binary64 fallback: factor (packed lower, in shared memory) and solve ----
    __syncthreads();
    for (int e = tid; e < n * n; e += T) {
        const int j = e / n, i = e - j * n;
        if (i >= j) Lp[pk(i, j, n)] = A[i + (long long)j * p.lda];
    }
    __syncthreads();
    if (tid == 0) s_flag = 0;
    __syncthreads();
    for (int j = 0; j < n; j++) {
        const double d = Lp[pk(j, j, n)];
        if (!(d > 0.0)) {
            if (tid == 0) s_flag = j + 1;
            break;
        }
        const double ljj = sqrt(d);
        const double rj = 1.0 / ljj;
        __syncthreads();
        if (tid == 0) Lp[pk(j, j, n)] = ljj;
        for (int i = j + 1 + tid; i < n; i += T) Lp[pk(i, j, n)] *= rj;
        __syncthreads();
        const int m = n - j - 1;
        for (int e = tid; e < m * m; e += T) {
            const int kk = e / m, ii = e - kk * m;
            const int i = j + 1 + ii, k = j + 1 + kk;
            if (i >= k) Lp[pk(i, k, n)] = fma(-Lp[pk(i, j, n)], Lp[pk(k, j, n)], Lp[pk(i, k, n)]);
        }
        __syncthreads();
    }
    __syncthreads();
    const int finfo = s_flag;
    if (finfo == 0) {
        for (int c = 0; c < p.nrhs; c++) {
            const double* b = B + (long long)c * p.ldb;
            for (int i = tid; i < n; i += T) xv[i] = b[i];
            __syncthreads();
            if (warp == 0) {
                for (int j = 0; j < n; j++) {
                    const double xj = xv[j] / Lp[pk(j, j, n)];
                    __syncwarp();
                    if (lane == 0) xv[j] = xj;
                    for (int i = j + 1 + lane; i < n; i += 32) xv[i] = fma(-Lp[pk(i, j, n)], xj, xv[i]);
                    __syncwarp();
                }
                for (int j = n - 1; j >= 0; j--) {
                    const double xj = xv[j] / Lp[pk(j, j, n)];
                    __syncwarp();
                    if (lane == 0) xv[j] = xj;
                    for (int i = lane; i < j; i += 32) xv[i] = fma(-Lp[pk(j, i, n)], xj, xv[i]);
                    __syncwarp();
                }
            }
            __syncthreads();
            double* x = X + (long long)c * p.ldx;
            for (int i = tid; i < n; i += T) x[i] = xv[i];
            __syncthreads();
        }
    }
    if (tid == 0) {
        if (p.iter) p.iter[q] = -1;
        if (p.info) p.info[q] = finfo;
    }
}

cudaError_t launch_dsposv(int n, int nrhs, MatRef A, int lda, MatRef B, int ldb, MatRef X, int ldx,
                          int* iter, int* info, double tol, int itmax, long long batch, cudaStream_t s) {
    if (batch == 0 || n == 0 || nrhs == 0) return cudaSuccess;
    SposvParams p;
    p.n = n; p.nrhs = nrhs; p.A = A; p.lda = lda; p.B = B; p.ldb = ldb; p.X = X; p.ldx = ldx;
    p.iter = iter; p.info = info; p.tol = tol; p.itmax = itmax; p.batch = batch;
    const size_t smem = sposv_smem_bytes(n);
    cudaError_t e = cudaFuncSetAttribute(dsposv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dsposv_kernel<<<(unsigned)batch, 256, smem, s>>>(p);
    count_launch();
    return cudaGetLastError();
}

}  // namespace bf

extern "C" int bf_dsposv_strided_batched(char uplo, int n, int nrhs, const double* A, int lda, long long strideA,
                                         const double* B, int ldb, long long strideB, double* X, int ldx,
                                         long long strideX, int* iter, int* info, double tol, int itmax,
                                         int batch, bf_stream_t stream) {
    const bool lo = (uplo == 'L' || uplo == 'l'), up = (uplo == 'U' || uplo == 'u');
    if (!(lo || up)) return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (lda < (n > 1 ? n : 1)) return -5;
    if (strideA < 0) return -6;
    if (ldb < (n > 1 ? n : 1)) return -8;
    if (ldx < (n > 1 ? n : 1)) return -11;
    if (batch < 0) return -17;
    if (batch > 1 && strideX < (long long)ldx * nrhs) return -12;
    if (!(tol >= 0.0)) return -15;
    if (itmax < 0) return -16;
    const bool work = n > 0 && nrhs > 0 && batch > 0;
    if (work && !A) return -4;
    if (work && !B) return -7;
    if (work && !X) return -10;
    if (up) return BF_ERR_NOT_SUPPORTED;
    if (n > BF_DSPOSV_NMAX) return BF_ERR_NOT_SUPPORTED;
    if (!work) return 0;
    cudaError_t e = bf::launch_dsposv(n, nrhs, bf::mat_strided(A, strideA), lda, bf::mat_strided(B, strideB), ldb,
                                      bf::mat_strided(X, strideX), ldx, iter, info, tol, itmax, batch,
                                      (cudaStream_t)stream);
    return e == cudaSuccess ? BF_SUCCESS : BF_ERR_CUDA;
}
