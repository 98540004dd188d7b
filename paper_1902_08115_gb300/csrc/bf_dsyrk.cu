// bf_dsyrk.cu -- batched FP64 dsyrk (section 3.1 "dsyrk") and the fused dsyrk + dpotrf of
// the paper's own API (section 5, "Riccati recursion").
//
// dsyrk: C <= alpha op(A) op(A)^T + beta C on the uplo triangle; op(A) = A (n x k) for 'N',
// A^T (A stored k x n) for 'T'.  The paper's point is that A and B of dgemm coincide, so
// one packed buffer serves both operands.  On the GPU the same reuse happens in L1: one
// thread computes one 4x4 tile of C that lies on or below (above, for 'U') the diagonal,
// reading both of its operand strips from the single array A.  Only the triangle's tiles are
// enumerated -- n/4 (n/4 + 1) / 2 per problem, flat over the batch -- so no thread works on
// the other triangle.  Consecutive threads take consecutive tiles of one tile row, so a warp
// shares one strip (broadcast) and reads the other as consecutive 4-row blocks.
//
// dsyrk + dpotrf, lower: C <= chol(C + A A^T).  For small orders in one pass: the lane
// Cholesky (one problem per thread, bf_lane.cuh) accumulates A A^T into the same register
// tiles as its own updates, so C + A A^T is never stored.  Larger orders run the tile dsyrk
// then dpotrf (measured faster: both halves are FP64-bound, so fusing saves only memory
// traffic that is not the bound, while the fused kernel's register count cuts occupancy).
#include "bf_internal.h"
#include "bf_lane.cuh"

namespace bf {

struct SyrkParams {
    int n, k;
    double alpha, beta;
    int mode;
    MatRef A;
    int lda;
    MatRef C;
    int ldc;
    long long batch;
    int tiles;  // 4x4 tiles of one triangle per problem
};

// Four consecutive entries x[i .. i+3] of a column (clamped to n - 1 at its end): 16-byte
// pieces from the first 16-byte boundary on.
__device__ __forceinline__ void col4(const double* x, int i, int n, double* o) {
    if (i + 4 <= n) {
        const double* p = x + i;
        if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
            const double2 a = ldg2(p), b = ldg2(p + 2);
            o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
        } else {
            const double2 a = ldg2(p + 1);
            o[0] = ldg(p); o[1] = a.x; o[2] = a.y; o[3] = ldg(p + 3);
        }
    } else {
#pragma unroll
        for (int r = 0; r < 4; r++) o[r] = ldg(x + imin(i + r, n - 1));
    }
}

// CIN: C's old values come from Cin (ld ldcin) rather than from C itself
template <bool TR, bool UP, bool CIN>
__global__ void __launch_bounds__(256) dsyrk_tile_kernel(SyrkParams p, MatRef Cin, int ldcin) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long q = g / p.tiles;
    if (q >= p.batch) return;
    const int t = (int)(g - q * p.tiles);
    // lower tiles numbered row block by row block: t = I (I + 1) / 2 + K, K <= I
    int I = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while ((I + 1) * (I + 2) / 2 <= t) I++;
    while (I * (I + 1) / 2 > t) I--;
    const int K = t - I * (I + 1) / 2;
    const int r0 = UP ? 4 * K : 4 * I, c0 = UP ? 4 * I : 4 * K;  // rows and columns of the C tile
    const int n = p.n;
    const double* A = p.A.ptr(q);
    double* C = p.C.mptr(q);

    double acc[4][4];
    if (p.mode == ACC_C || p.mode == ACC_BC) {
#pragma unroll
        for (int b = 0; b < 4; b++) {
            double col[4];
            if constexpr (CIN) col4(Cin.ptr(q) + (long long)imin(c0 + b, n - 1) * ldcin, r0, n, col);
            else col4(C + (long long)imin(c0 + b, n - 1) * p.ldc, r0, n, col);  // the other triangle is read, not used
#pragma unroll
            for (int a = 0; a < 4; a++) acc[a][b] = (p.mode == ACC_BC) ? p.beta * col[a] : col[a];
        }
    } else {
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++) acc[a][b] = 0.0;
    }
    int ri[4], ci[4];
#pragma unroll
    for (int a = 0; a < 4; a++) {
        ri[a] = imin(r0 + a, n - 1);
        ci[a] = imin(c0 + a, n - 1);
    }
#pragma unroll 2
    for (int pp = 0; pp < p.k; pp++) {
        double x[4], y[4];
        if (TR) {  // op(A)(i, pp) = A[pp + i lda]: one word per row
#pragma unroll
            for (int a = 0; a < 4; a++) {
                x[a] = ldg(A + pp + (long long)ri[a] * p.lda);
                y[a] = ldg(A + pp + (long long)ci[a] * p.lda);
            }
        } else {
            col4(A + (long long)pp * p.lda, r0, n, x);
            col4(A + (long long)pp * p.lda, c0, n, y);
        }
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++) acc[a][b] = fma(x[a], y[b], acc[a][b]);
    }
#pragma unroll
    for (int b = 0; b < 4; b++) {
        const int j = c0 + b;
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int i = r0 + a;
            if (i < n && j < n && (UP ? i <= j : i >= j)) {
                double* cp = C + i + (long long)j * p.ldc;
                double v = acc[a][b];
                if constexpr (CIN) {
                    if (p.mode == ACC_GEN)
                        v = (p.beta == 0.0) ? p.alpha * v : fma(p.alpha, v, p.beta * Cin.ptr(q)[i + (long long)j * ldcin]);
                } else {
                    if (p.mode == ACC_GEN) v = (p.beta == 0.0) ? p.alpha * v : fma(p.alpha, v, p.beta * *cp);
                }
                *cp = v;
            }
        }
    }
}

// C <= beta * C on the uplo triangle (alpha == 0 or k == 0); beta == 0 writes zeros
__global__ void dsyrk_scale_kernel(int n, int upper, double beta, MatRef C, int ldc, long long batch) {
    const long long per = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per * batch;
         e += (long long)gridDim.x * blockDim.x) {
        const long long q = e / per;
        const long long r = e - q * per;
        const int j = (int)(r / n), i = (int)(r - (long long)j * n);
        if (upper ? i > j : i < j) continue;
        double* cp = C.mptr(q) + i + (long long)j * ldc;
        *cp = (beta == 0.0) ? 0.0 : beta * *cp;
    }
}

cudaError_t launch_dsyrk(int upper, int trans, int n, int k, double alpha, MatRef A, int lda, double beta,
                         MatRef C, int ldc, long long batch, cudaStream_t s, const MatRef* Cin, int ldcin) {
    if (n == 0 || batch == 0) return cudaSuccess;
    if (Cin && (alpha == 0.0 || k == 0)) return cudaErrorInvalidValue;  // not needed by any caller
    if (alpha == 0.0 || k == 0) {
        if (beta == 1.0) return cudaSuccess;
        long long total = (long long)n * n * batch;
        int blocks = (int)((total + 255) / 256);
        if (blocks > kSMs * 64) blocks = kSMs * 64;
        dsyrk_scale_kernel<<<blocks, 256, 0, s>>>(n, upper, beta, C, ldc, batch);
        count_launch();
        return cudaGetLastError();
    }
    SyrkParams p;
    p.n = n; p.k = k; p.alpha = alpha; p.beta = beta;
    p.mode = acc_mode(alpha, beta);
    p.A = A; p.lda = lda; p.C = C; p.ldc = ldc; p.batch = batch;
    const MatRef cin = Cin ? *Cin : C;
    const int nI = (n + 3) / 4;
    p.tiles = nI * (nI + 1) / 2;
    const long long threads = batch * (long long)p.tiles;
    const int T = spread_block(threads, 256);
    const unsigned blocks = (unsigned)((threads + T - 1) / T);
#define BF_SYRK_LAUNCH(TR_, UP_)                                                              \
    if (Cin) dsyrk_tile_kernel<TR_, UP_, true><<<blocks, T, 0, s>>>(p, cin, ldcin);          \
    else dsyrk_tile_kernel<TR_, UP_, false><<<blocks, T, 0, s>>>(p, cin, ldcin);
    if (trans) {
        if (upper) { BF_SYRK_LAUNCH(true, true) } else { BF_SYRK_LAUNCH(true, false) }
    } else {
        if (upper) { BF_SYRK_LAUNCH(false, true) } else { BF_SYRK_LAUNCH(false, false) }
    }
#undef BF_SYRK_LAUNCH
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ fused dsyrk + dpotrf
struct SyrkPotrfParams {
    int n, k;
    MatRef A;
    int lda;
    MatRef C;
    int ldc;
    long long batch;
    int* info;
    int stage;    // >= 0: info is the recursion's stage-tagged status (written only while 0)
};

// C(i, j) = Cin(i, j) on the lower triangle of every problem: flat over the batch, consecutive
// threads on consecutive rows of a column (coalesced)
__global__ void copy_lower_kernel(int n, MatRef Cin, int ldcin, MatRef C, int ldc, long long batch) {
    const long long per = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per * batch;
         e += (long long)gridDim.x * blockDim.x) {
        const long long q = e / per;
        const int r = (int)(e - q * per), j = r / n, i = r - j * n;
        if (i >= j) C.mptr(q)[i + (long long)j * ldc] = Cin.ptr(q)[i + (long long)j * ldcin];
    }
}

template <int R, int U>
__global__ void __launch_bounds__(256) dsyrk_dpotrf_lane_kernel(SyrkPotrfParams p) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= p.batch) return;
    const SyrkOp<GAccP> y{GAccP{const_cast<double*>(p.A.ptr(q)), p.lda}};  // read only
    const int info = potrf_lane<R, U>(GAccP{p.C.mptr(q), p.ldc}, p.n, y, p.k);
    if (p.info) {
        if (p.stage < 0) p.info[q] = info;
        else if (info != 0 && p.info[q] == 0) p.info[q] = 1000 * p.stage + info;
    }
}

cudaError_t launch_dsyrk_dpotrf(int n, int k, MatRef A, int lda, MatRef C, int ldc, long long batch, int* info,
                                cudaStream_t s, const MatRef* Cin, int ldcin, int* merged, int stage) {
    if (batch == 0) return cudaSuccess;
    PotrfConfig cfg = choose_potrf(n, ldc, batch);
    // the size switch of the fused routine: the one-pass lane kernel wins for small orders
    // (n <= 12: the rank-k update is latency-bound on its own); above that the coalesced
    // tile dsyrk then the lane/blocked dpotrf is faster on this GPU, since the FP64 pipe, not
    // memory, bounds both halves and the fused kernel's registers cut its occupancy
    if (n == 0 || n > 12 || cfg.variant == VAR_BLOCKED || cfg.variant == VAR_GROUP) {
        cudaError_t e = launch_dsyrk(0, 0, n, k, 1.0, A, lda, 1.0, C, ldc, batch, s, Cin, ldcin);
        if (e != cudaSuccess) return e;
        e = launch_dpotrf(n, C, ldc, batch, info, cfg, s);
        if (e != cudaSuccess || !merged) return e;
        return launch_merge_stage_info(info, merged, stage, batch, s);
    }
    SyrkPotrfParams p;
    p.n = n; p.k = k; p.A = A; p.lda = lda; p.C = C; p.ldc = ldc; p.batch = batch;
    p.info = merged ? merged : info;
    p.stage = merged ? stage : -1;
    if (Cin) {  // a coalesced copy first: the lane kernel's own loads would be one problem per lane
        const long long total = (long long)n * n * batch;
        long long blocks = (total + 255) / 256;
        if (blocks > kSMs * 32) blocks = kSMs * 32;
        copy_lower_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, *Cin, ldcin, C, ldc, batch);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int T = cfg.T > 0 ? (cfg.T < 256 ? cfg.T : 256) : 64;
    const unsigned blocks = (unsigned)((batch + T - 1) / T);
    if (cfg.rows == 8) {
        if (cfg.unroll == 1) dsyrk_dpotrf_lane_kernel<8, 1><<<blocks, T, 0, s>>>(p);
        else dsyrk_dpotrf_lane_kernel<8, 2><<<blocks, T, 0, s>>>(p);
    } else {
        if (cfg.unroll == 1) dsyrk_dpotrf_lane_kernel<4, 1><<<blocks, T, 0, s>>>(p);
        else dsyrk_dpotrf_lane_kernel<4, 2><<<blocks, T, 0, s>>>(p);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace bf
