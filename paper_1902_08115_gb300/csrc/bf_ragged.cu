// bf_ragged.cu -- ragged batches: every problem has its own order n_b.  One
// persistent kernel, captured in a CUDA graph, factors each SPD matrix
// (dpotrf, lower, section 3.1) and solves its right-hand sides (dpotrs).
//
// Work items come from a device queue (one atomic counter, no waiting between
// CTAs), ordered by decreasing cost so the largest problems start first:
//   BIG items  (n_b > lane_max, n_b <= 256): one problem per CTA, left-looking by
//     16-column panels: the panel is updated with the factored columns (read back from
//     the matrix through L1/L2) on 4x4 register tiles, its diagonal block is factored by
//     one warp (pivots via rsqrt), the rows below by all threads; the right-hand sides
//     follow panel by panel (forward substitution), then a warp-per-right-hand-side
//     backward substitution.  Only the panel lives in shared memory, so several
//     problems share an SM and cover each other's serial phases.
//   LANE items (n_b <= lane_max): blockDim problems per CTA, one per thread,
//     sorted so a warp's problems have (nearly) equal order, using the same
//     lane Cholesky as the uniform path.
// The threshold lane_max and the CTA size are picked by the autotuner.
#include <algorithm>
#include <numeric>
#include <vector>

#include "bf_internal.h"
#include "bf_lane.cuh"
#include "../../include/bfgpu.h"

namespace bf {

struct RaggedParams {
    const int* n;            // order of each problem, in queue order
    const long long* offS;   // element offset of each matrix (ld = n)
    const long long* offB;   // element offset of each right-hand-side block (ld = n)
    const int* orig;         // original index (for info)
    double* S;
    double* B;
    int* info;
    int nrhs;
    int nbig;                // problems [0, nbig) are BIG items
    int nprob;
    int nitems;
    unsigned int* counter;
};

// --------------------------------------------------------------------------- BIG: one problem per CTA
#define BF_BIG_NB 16
#define BF_BIG_NMAX 256  // backward substitution keeps x in 8 registers per lane

// Element (i, k) of the factored matrix: column-major with leading dimension ld, or, with TR,
// of its transpose (the upper Cholesky A = U^T U is the lower one of the transposed view).
template <bool TR>
__device__ __forceinline__ long long bidx(int i, int k, int ld) {
    return TR ? k + (long long)i * ld : i + (long long)k * ld;
}

// Four consecutive rows i..i+3 of column k of a problem in global memory (leading dimension
// ld, rows clamped to n - 1): two 16-byte loads when the strip starts on a 16-byte boundary,
// one 16-byte load between two single words when it starts 8 bytes past one; single words
// along a row of the stored matrix for the transposed view.
template <bool TR>
__device__ __forceinline__ void big_strip4(const double* S, int ld, int n, int i, int k, double* o) {
    if (TR) {
#pragma unroll
        for (int a = 0; a < 4; a++) o[a] = S[bidx<TR>(imin(i + a, n - 1), k, ld)];
        return;
    }
    const double* p = S + i + (long long)k * ld;
    if (i + 4 <= n) {
        if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
            const double2 x = reinterpret_cast<const double2*>(p)[0], y = reinterpret_cast<const double2*>(p)[1];
            o[0] = x.x; o[1] = x.y; o[2] = y.x; o[3] = y.y;
        } else {
            const double2 x = reinterpret_cast<const double2*>(p + 1)[0];
            o[0] = p[0]; o[1] = x.x; o[2] = x.y; o[3] = p[3];
        }
    } else {
#pragma unroll
        for (int a = 0; a < 4; a++) o[a] = S[imin(i + a, n - 1) + (long long)k * ld];
    }
}

// Tile t of a panel's lower tiles, column block by column block: column block K holds the
// row blocks I = K .. nI-1 (consecutive t: consecutive row blocks of one column block).
__device__ __forceinline__ void big_tile_index(int t, int nI, int& K, int& I) {
    K = 0;
    while (t >= nI - K) {
        t -= nI - K;
        K++;
    }
    I = K + t;
}

// Left-looking Cholesky by 16-column panels with the panel in shared memory and the
// factored columns in global memory (read back through L1/L2), so a CTA holds about
// 17 n doubles and several problems share an SM, each filling the FP64 pipes while
// another is in a serial phase.  Per panel J (section 3.2.1's dgemm loop + edges, at
// CTA scale):
//   (1) W = A(J:n, J:J+nb) - L(J:n, 0:J) L(J:J+nb, 0:J)^T on 4x4 register tiles
//       (lower tiles only), and the right-hand-side rows J..J+nb minus L(J:J+nb, 0:J) Y(0:J);
//   (2) one warp factors W's diagonal block (pivots via rsqrt);
//   (3) every thread: one row of the panel below, L(i,:) = W(i,:) L_JJ^{-T}, written to the
//       matrix, and the diagonal block written back; the last warp solves
//       Y(J:J+nb) = L_JJ^{-1} (rows J..J+nb) -- the forward substitution, panel by panel.
// Then the backward substitution L^T X = Y, one warp per right-hand side.  The matrix S has
// leading dimension lds, the r right-hand sides Bq leading dimension n; returns the LAPACK
// info (every thread).  Shared memory: 8 (16 n + n r + n + 16 blockDim) bytes at sm.
template <bool TR>
__device__ int big_core(int n, double* S, int lds, double* Bq, int r, double* sm) {
    const int tid = threadIdx.x, T = blockDim.x, warp = tid >> 5, lane = tid & 31;
    double* W = sm;                            // panel: W[i + c n], i = row - J, c < 16
    double* X = sm + (size_t)BF_BIG_NB * n;    // n x nrhs right-hand sides
    double* rinv = X + (size_t)n * r;          // reciprocal pivots
    __shared__ int s_fail;
    for (int e = tid; e < n * r; e += T) X[e] = Bq[e];
    if (tid == 0) s_fail = 0;
    __syncthreads();

    for (int J = 0; J < n; J += BF_BIG_NB) {
        const int nb = imin(BF_BIG_NB, n - J), m = n - J;
        // (1) panel update: tile (I, K) covers rows J+4I.., columns J+4K..; consecutive
        //     threads take consecutive row blocks of one column block (the L(J+4K.., k)
        //     operand is then the same for the whole warp).  The tiles go out in rounds of
        //     T; the rem tiles of the last, partial round (all of them in the late panels:
        //     few rows, long k loops) have their k range split sp ways, so the idle lanes of
        //     a mostly empty round turn into work; the partial sums are added in a fixed
        //     order, so the result is reproducible.
        {
            const int nI = (m + 3) / 4, nK = (nb + 3) / 4;
            const int tiles = nI * nK - nK * (nK - 1) / 2;  // tiles on or below the diagonal block
            // The last round: either every one of its rem tiles split sp ways, or whole warps of
            // unsplit tiles and only the rem % 32 tiles that would leave a warp part-empty split
            // over the remaining threads -- whichever leaves fewer idle lanes in issued FP64
            // instructions (a warp's instruction costs the SM's FP64 unit a full slot whatever
            // its active lanes, and its lanes all wait for its longest k range).
            const int full = tiles / T * T, rem = tiles - full;
            int unsplit = 0, tail = rem, sp = rem ? imax(1, imin(T / rem, J / 8)) : 1;
            if (rem > 32 && (rem & 31)) {
                const int t2 = rem & 31, sp2 = imax(1, imin((T - (rem - t2)) / t2, J / 8));
                const int l1 = (rem * sp) & 31, l2 = (t2 * sp2) & 31;
                const long long w1 = (long long)(l1 ? 32 - l1 : 0) * (J / sp);
                const long long w2 = (long long)(l2 ? 32 - l2 : 0) * (J / sp2);
                if (w2 < w1) {
                    unsplit = rem - t2;
                    tail = t2;
                    sp = sp2;
                }
            }
            const int base = full + unsplit;  // the first split tile
            double* part = rinv + n;          // [sp][16][tail] partial sums, only when sp > 1
            for (int u = tid; u < base + tail * sp; u += T) {
                int t = u, z = 0;
                if (u >= base) {
                    z = (u - base) / tail;
                    t = u - z * tail;
                }
                const bool split = u >= base && sp > 1;
                int K, I;
                big_tile_index(t, nI, K, I);
                const int i0 = J + 4 * I, k0 = J + 4 * K;
                const int klo = split ? (J * z) / sp : 0, khi = split ? (J * (z + 1)) / sp : J;
                double acc[4][4];
                if (z == 0) {
#pragma unroll
                    for (int b = 0; b < 4; b++) {
                        double col[4];
                        big_strip4<TR>(S, lds, n, i0, imin(k0 + b, n - 1), col);  // upper entries unused
#pragma unroll
                        for (int a = 0; a < 4; a++) acc[a][b] = col[a];
                    }
                } else {
#pragma unroll
                    for (int a = 0; a < 4; a++)
#pragma unroll
                        for (int b = 0; b < 4; b++) acc[a][b] = 0.0;
                }
#pragma unroll 2
                for (int k = klo; k < khi; k++) {
                    double li[4], lk[4];
                    big_strip4<TR>(S, lds, n, i0, k, li);
#pragma unroll
                    for (int b = 0; b < 4; b++) lk[b] = S[bidx<TR>(imin(k0 + b, n - 1), k, lds)];
#pragma unroll
                    for (int a = 0; a < 4; a++)
#pragma unroll
                        for (int b = 0; b < 4; b++) acc[a][b] = fma(-li[a], lk[b], acc[a][b]);
                }
                if (!split) {
#pragma unroll
                    for (int b = 0; b < 4; b++) {
                        const int c = 4 * K + b;
                        if (c >= nb) continue;
#pragma unroll
                        for (int a = 0; a < 4; a++)
                            if (4 * I + a < m) W[4 * I + a + c * n] = acc[a][b];
                    }
                } else {
#pragma unroll
                    for (int a = 0; a < 4; a++)
#pragma unroll
                        for (int b = 0; b < 4; b++) part[(z * 16 + a * 4 + b) * tail + (t - base)] = acc[a][b];
                }
            }
            for (int e = T - 1 - tid; e < nb * r; e += T) {  // the last threads, fewest tiles
                const int c = e % nb, rr = e / nb;
                double s = X[J + c + (size_t)rr * n];
                for (int k = 0; k < J; k++) s = fma(-S[bidx<TR>(J + c, k, lds)], X[k + (size_t)rr * n], s);
                X[J + c + (size_t)rr * n] = s;
            }
            if (sp > 1) {
                __syncthreads();
                for (int e = tid; e < 16 * tail; e += T) {
                    const int ab = e / tail, tt = e - ab * tail;
                    int K, I;
                    big_tile_index(base + tt, nI, K, I);
                    const int c = 4 * K + (ab & 3), i = 4 * I + (ab >> 2);
                    if (c >= nb || i >= m) continue;
                    double v = part[ab * tail + tt];
                    for (int z = 1; z < sp; z++) v += part[(z * 16 + ab) * tail + tt];
                    W[i + c * n] = v;
                }
            }
        }
        __syncthreads();
        // (2) the diagonal block, warp-synchronous in warp 0.  This runs on one warp while the
        //     CTA's others wait, and every FP64 instruction of it costs the SM's FP64 unit a full
        //     slot whatever its active lanes, so it issues as few as it can: the pivot test on
        //     the bits (d > 0: 0 < bits <= the bits of +inf, the same predicate for every double),
        //     l_cc = d rs and the column's scale as one multiply (lane c holds the diagonal), and
        //     the update over the trailing triangle's entries only.
        if (warp == 0) {
            for (int c = 0; c < nb; c++) {
                const double d = W[c + c * n];
                const long long db = __double_as_longlong(d);
                if (!(db > 0 && db <= 0x7ff0000000000000ll)) {  // the same value in every lane
                    if (lane == 0) s_fail = J + c + 1;
                    break;
                }
                const double rs = rsqrt(d);
                __syncwarp();
                if (lane == 0) rinv[J + c] = rs;
                if (lane >= c && lane < nb) W[lane + c * n] *= rs;  // lane c: d rs
                __syncwarp();
                // entry e of the w x w trailing triangle, row by row: e = ii (ii + 1) / 2 + kk
                const int w = nb - c - 1;
                for (int e = lane; e < w * (w + 1) / 2; e += 32) {
                    int ii = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
                    if ((ii + 1) * (ii + 2) / 2 <= e) ii++;
                    if (ii * (ii + 1) / 2 > e) ii--;
                    const int kk = e - ii * (ii + 1) / 2;
                    const int i = c + 1 + ii, k = c + 1 + kk;
                    W[i + k * n] = fma(-W[i + c * n], W[k + c * n], W[i + k * n]);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (s_fail) break;  // written before the barrier: the same in every thread
        // (3) rows below the diagonal block, the diagonal block itself, and Y of the block's rows
        for (int i = nb + tid; i < m; i += T) {
            double x[BF_BIG_NB];
#pragma unroll
            for (int c = 0; c < BF_BIG_NB; c++) x[c] = (c < nb) ? W[i + c * n] : 0.0;
#pragma unroll
            for (int c = 0; c < BF_BIG_NB; c++) {
                if (c < nb) {
#pragma unroll
                    for (int c2 = 0; c2 < c; c2++) x[c] = fma(-x[c2], W[c + c2 * n], x[c]);
                    x[c] *= rinv[J + c];
                    S[bidx<TR>(J + i, J + c, lds)] = x[c];
                }
            }
        }
        for (int e = tid; e < nb * nb; e += T) {
            const int c = e / nb, i = e - c * nb;
            if (i >= c) S[bidx<TR>(J + i, J + c, lds)] = W[i + c * n];
        }
        if (warp == (T >> 5) - 1) {
            // Y(J:J+nb, :) = L_JJ^{-1} (rows J..J+nb), column-oriented by the last warp: step c
            // scales row J+c of every right-hand side, then its lanes update the rows below
            for (int c = 0; c < nb; c++) {
                for (int e = lane; e < r; e += 32) X[J + c + (size_t)e * n] *= rinv[J + c];
                __syncwarp();
                const int w = nb - c - 1;
                for (int e = lane; e < w * r; e += 32) {
                    const int i = c + 1 + e % w, rr = e / w;
                    X[J + i + (size_t)rr * n] = fma(-W[i + c * n], X[J + c + (size_t)rr * n], X[J + i + (size_t)rr * n]);
                }
                __syncwarp();
            }
        }
        __syncthreads();  // the panel's columns of L (global) and Y (shared) are complete
    }
    const int fail = s_fail;
    if (fail == 0) {
        // backward substitution L^T x = y, one warp per right-hand side: lane l holds x_i for
        // i = l, l + 32, ...; x_j is broadcast from its lane, then every lane updates its
        // x_i, i < j, with L(j, i); the next step's L(j - 1, i) is loaded a step ahead
        constexpr int NS = BF_BIG_NMAX / 32;
        for (int rr = warp; rr < r; rr += T >> 5) {
            double* y = X + (size_t)rr * n;
            double xr[NS], ln[NS];
#pragma unroll
            for (int s = 0; s < NS; s++) {
                const int i = lane + 32 * s;
                xr[s] = (i < n) ? y[i] : 0.0;
                ln[s] = (i < n - 1) ? S[bidx<TR>(n - 1, i, lds)] : 0.0;
            }
#pragma unroll
            for (int s = NS - 1; s >= 0; s--) {
                if (32 * s >= n) continue;
                for (int lj = imin(31, n - 1 - 32 * s); lj >= 0; lj--) {
                    const int j = 32 * s + lj;
                    double lc[NS];
#pragma unroll
                    for (int s2 = 0; s2 <= s; s2++) {
                        const int i = lane + 32 * s2;
                        lc[s2] = ln[s2];
                        ln[s2] = (i < j - 1) ? S[bidx<TR>(j - 1, i, lds)] : 0.0;
                    }
                    const double xj = __shfl_sync(0xffffffffu, xr[s], lj) * rinv[j];
                    if (lane == lj) xr[s] = xj;
#pragma unroll
                    for (int s2 = 0; s2 <= s; s2++) {
                        const int i = lane + 32 * s2;
                        if (i < j) xr[s2] = fma(-lc[s2], xj, xr[s2]);
                    }
                }
            }
#pragma unroll
            for (int s = 0; s < NS; s++)
                if (lane + 32 * s < n) Bq[lane + 32 * s + (size_t)rr * n] = xr[s];
        }
    }
    __syncthreads();
    return fail;
}

__device__ void big_problem(const RaggedParams& p, int q, double* sm) {
    const int n = p.n[q];
    const int fail = big_core<false>(n, p.S + p.offS[q], n, p.B + p.offB[q], p.nrhs, sm);
    if (threadIdx.x == 0 && p.info) p.info[p.orig[q]] = fail;
}

// --------------------------------------------------------------------------- LANE: one problem per thread
__device__ void lane_problem(const RaggedParams& p, int q) {
    const int n = p.n[q];
    double* S = p.S + p.offS[q];
    double* Bq = p.B + p.offB[q];
    const int info = potrf_lane_global<4, 2>(S, n, n);
    if (info == 0) {
        for (int c = 0; c < p.nrhs; c++) {
            double* b = Bq + (long long)c * n;
            for (int j = 0; j < n; j++) {
                const double yj = b[j] / S[j + (long long)j * n];
                b[j] = yj;
                for (int i = j + 1; i < n; i++) b[i] = fma(-S[i + (long long)j * n], yj, b[i]);
            }
            for (int j = n - 1; j >= 0; j--) {
                double s = b[j];
                for (int i = j + 1; i < n; i++) s = fma(-S[i + (long long)j * n], b[i], s);
                b[j] = s / S[j + (long long)j * n];
            }
        }
    }
    if (p.info) p.info[p.orig[q]] = info;
}

// --------------------------------------------------------------------------- uniform batches, one problem per CTA
// dpotrf of a uniform batch with too few problems to fill the GPU one problem per thread (a
// warp issues one FP64 instruction every 64 cycles, so the lane kernels need ~20,000
// problems): the BIG items' left-looking Cholesky, one problem per CTA, any leading
// dimension, no right-hand sides.  CTAs stride over the batch.
template <bool TR>
__global__ void __launch_bounds__(128, 6) dpotrf_cta_kernel(int n, MatRef A, int lda, long long batch, int* info) {
    extern __shared__ __align__(16) double sm_cta[];
    for (long long q = blockIdx.x; q < batch; q += gridDim.x) {
        const int fail = big_core<TR>(n, A.mptr(q), lda, nullptr, 0, sm_cta);
        if (threadIdx.x == 0 && info) info[q] = fail;
    }
}

cudaError_t launch_dpotrf_cta(int n, MatRef A, int lda, long long batch, int* info, cudaStream_t s, int upper) {
    const int T = 128;
    const size_t smem = sizeof(double) * ((size_t)(BF_BIG_NB + 1) * n + 16 * (size_t)T);
    if (smem + kStaticSmemSlack > 48 * 1024) {
        cudaError_t e = upper ? cudaFuncSetAttribute(dpotrf_cta_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem)
                              : cudaFuncSetAttribute(dpotrf_cta_kernel<false>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const long long cap = kSMs * 16;
    const unsigned grid = (unsigned)(batch < cap ? batch : cap);
    if (upper) dpotrf_cta_kernel<true><<<grid, T, smem, s>>>(n, A, lda, batch, info);
    else dpotrf_cta_kernel<false><<<grid, T, smem, s>>>(n, A, lda, batch, info);
    count_launch();
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- variable-size batches
// dpotrf 'L' of a variable-size batch: problem q has order n[q] and leading dimension lda[q]
// (device arrays) at Aarray[q].  An illegal problem (n < 0 or above max_n: -2; lda < max(1, n):
// -4) is skipped with info = that negative position.  Orders up to 32: one problem per
// thread (the lane Cholesky, in place); larger: one problem per CTA (the left-looking CTA
// Cholesky above), CTAs striding over the batch.
__device__ __forceinline__ int vpotrf_check(int n, int lda, int max_n) {
    if (n < 0 || n > max_n) return -2;
    if (lda < (n > 1 ? n : 1)) return -4;
    return 0;
}

template <bool TR>
__global__ void __launch_bounds__(128) dpotrf_vbatched_lane_kernel(const int* n, double* const* A, const int* lda,
                                                                 int* info, long long batch, int max_n) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= batch) return;
    const int nq = n[q], ldq = lda[q];
    int r = vpotrf_check(nq, ldq, max_n);
    if (r == 0 && nq > 0)
        r = TR ? potrf_lane<4, 2>(GAccT{A[q], ldq}, nq) : potrf_lane_global<4, 2>(A[q], ldq, nq);
    if (info) info[q] = r;
}

template <bool TR>
__global__ void __launch_bounds__(128, 6) dpotrf_vbatched_cta_kernel(const int* n, double* const* A, const int* lda,
                                                                int* info, long long batch, int max_n) {
    extern __shared__ __align__(16) double sm_v[];
    for (long long q = blockIdx.x; q < batch; q += gridDim.x) {
        const int nq = n[q], ldq = lda[q];
        int r = vpotrf_check(nq, ldq, max_n);  // the same in every thread
        if (r == 0 && nq > 0) r = big_core<TR>(nq, A[q], ldq, nullptr, 0, sm_v);
        if (threadIdx.x == 0 && info) info[q] = r;
    }
}

cudaError_t launch_dpotrf_vbatched(const int* n, double* const* A, const int* lda, int* info, long long batch,
                                   int max_n, cudaStream_t s, int upper) {
    if (batch == 0) return cudaSuccess;
    if (max_n <= 32) {  // one problem per thread; small batches in smaller CTAs, over every SM
        const int T = spread_block(batch, 128);
        const unsigned blocks = (unsigned)((batch + T - 1) / T);
        if (upper) dpotrf_vbatched_lane_kernel<true><<<blocks, T, 0, s>>>(n, A, lda, info, batch, max_n);
        else dpotrf_vbatched_lane_kernel<false><<<blocks, T, 0, s>>>(n, A, lda, info, batch, max_n);
        count_launch();
        return cudaGetLastError();
    }
    const int T = 128;
    const size_t smem = sizeof(double) * ((size_t)(BF_BIG_NB + 1) * max_n + 16 * (size_t)T);
    if (smem + kStaticSmemSlack > 48 * 1024) {
        cudaError_t e = upper ? cudaFuncSetAttribute(dpotrf_vbatched_cta_kernel<true>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                              : cudaFuncSetAttribute(dpotrf_vbatched_cta_kernel<false>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    // one CTA per problem: the orders differ, so a fixed share of the batch per CTA (a
    // grid-stride loop) leaves the SMs unequal work; CTAs issued as SM slots free up balance
    // it (200,000 problems, n log-uniform in [2, 200]: 716 -> 819 GFLOP/s on GB300)
    const long long cap = 0x7fffffffLL;
    const unsigned grid = (unsigned)(batch < cap ? batch : cap);
    if (upper) dpotrf_vbatched_cta_kernel<true><<<grid, T, smem, s>>>(n, A, lda, info, batch, max_n);
    else dpotrf_vbatched_cta_kernel<false><<<grid, T, smem, s>>>(n, A, lda, info, batch, max_n);
    count_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(512) ragged_persistent_kernel(RaggedParams p) {
    extern __shared__ double smem[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(p.counter, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= p.nitems) break;
        if (item < p.nbig) {
            big_problem(p, item, smem);
        } else {
            const int q = p.nbig + (item - p.nbig) * (int)blockDim.x + (int)threadIdx.x;
            if (q < p.nprob) lane_problem(p, q);
        }
    }
}

size_t ragged_smem_bytes(int nmax, int nrhs, int threads) {
    // BIG items: a 16-column panel, the right-hand sides, the reciprocal pivots and the
    // split-k partial sums (at most 16 per thread)
    if (nmax == 0) return 0;
    return sizeof(double) * ((size_t)BF_BIG_NB * nmax + (size_t)nmax * nrhs + nmax + 16 * (size_t)threads);
}

}  // namespace bf

// ----------------------------------------------------------------------------- plan
struct bf_ragged_plan_st {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bf::RaggedParams p;
    int threads, blocks;
    size_t smem;
};

extern "C" size_t bf_ragged_workspace_bytes(int batch) {
    // n, orig (int) + offS, offB (int64) per problem, one counter, 256-byte alignment slack
    return (size_t)batch * (2 * sizeof(int) + 2 * sizeof(long long)) + 4 * 256;
}

extern "C" int bf_ragged_potrf_potrs_plan_create(int batch, const int* n_host, int nrhs, double* S,
                                                 const long long* offS_host, double* B,
                                                 const long long* offB_host, int* info, void* workspace,
                                                 size_t workspace_bytes, int lane_max, int threads,
                                                 bf_stream_t stream, bf_ragged_plan_t* plan) {
    if (batch < 0) return -1;
    if (batch > 0 && !n_host) return -2;
    if (nrhs < 0 || nrhs > 64) return -3;
    if (batch > 0 && !S) return -4;
    if (batch > 0 && !offS_host) return -5;
    if (batch > 0 && nrhs > 0 && !B) return -6;
    if (batch > 0 && nrhs > 0 && !offB_host) return -7;
    if (workspace_bytes < bf_ragged_workspace_bytes(batch)) return -10;
    if (batch > 0 && !workspace) return -9;
    if (lane_max < 0) return -11;
    if (threads != 64 && threads != 128 && threads != 256 && threads != 512) return -12;
    if (!plan) return -14;
    int nmax = 0;
    for (int b = 0; b < batch; b++) {
        if (n_host[b] < 0) return -2;
        nmax = std::max(nmax, n_host[b]);
    }
    const size_t smem = bf::ragged_smem_bytes(nmax > lane_max ? nmax : 0, nrhs, threads);
    if (smem > 227 * 1024 || (nmax > lane_max && nmax > BF_BIG_NMAX)) return BF_ERR_NOT_SUPPORTED;
    // queue order: BIG problems by decreasing order, then LANE problems by decreasing order
    std::vector<int> order(batch);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n_host[a] > n_host[b]; });
    int nbig = 0;
    while (nbig < batch && n_host[order[nbig]] > lane_max) nbig++;
    std::vector<int> nq(batch), orig(batch);
    std::vector<long long> oS(batch), oB(batch);
    for (int i = 0; i < batch; i++) {
        const int b = order[i];
        nq[i] = n_host[b];
        orig[i] = b;
        oS[i] = offS_host[b];
        oB[i] = nrhs ? offB_host[b] : 0;
    }
    auto align = [](size_t x) { return (x + 255) / 256 * 256; };
    char* w = (char*)workspace;
    size_t o = 0;
    unsigned int* counter = (unsigned int*)(w + o);
    o = align(o + sizeof(unsigned int));
    int* dn = (int*)(w + o);
    o = align(o + sizeof(int) * batch);
    int* dorig = (int*)(w + o);
    o = align(o + sizeof(int) * batch);
    long long* doS = (long long*)(w + o);
    o = align(o + sizeof(long long) * batch);
    long long* doB = (long long*)(w + o);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (batch > 0) {
        e = cudaMemcpyAsync(dn, nq.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dorig, orig.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(doS, oS.data(), sizeof(long long) * batch, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(doB, oB.data(), sizeof(long long) * batch, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors go out of scope
        if (e != cudaSuccess) return BF_ERR_CUDA;
    }
    bf_ragged_plan_st* pl = new bf_ragged_plan_st();
    pl->p.n = dn;
    pl->p.offS = doS;
    pl->p.offB = doB;
    pl->p.orig = dorig;
    pl->p.S = S;
    pl->p.B = B;
    pl->p.info = info;
    pl->p.nrhs = nrhs;
    pl->p.nbig = nbig;
    pl->p.nprob = batch;
    pl->p.nitems = nbig + (batch - nbig + threads - 1) / threads;
    pl->p.counter = counter;
    pl->threads = threads;
    pl->smem = smem;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (smem + bf::kStaticSmemSlack > 48 * 1024 &&
        cudaFuncSetAttribute(bf::ragged_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
        delete pl;
        return BF_ERR_CUDA;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bf::ragged_persistent_kernel, threads, smem) !=
            cudaSuccess ||
        per_sm < 1) {
        delete pl;
        return BF_ERR_CUDA;
    }
    pl->blocks = sms * per_sm;
    // capture: reset the queue counter, then the persistent launch
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        delete pl;
        return BF_ERR_CUDA;
    }
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(counter, 0, sizeof(unsigned int), cs);
        bf::ragged_persistent_kernel<<<pl->blocks, threads, smem, cs>>>(pl->p);
        e = cudaStreamEndCapture(cs, &pl->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        delete pl;
        return BF_ERR_CUDA;
    }
    *plan = pl;
    return BF_SUCCESS;
}

extern "C" int bf_ragged_plan_launch(bf_ragged_plan_t plan, bf_stream_t stream) {
    if (!plan) return -1;
    if (plan->p.nprob == 0) return BF_SUCCESS;
    cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
    bf::count_launch();
    return e == cudaSuccess ? BF_SUCCESS : BF_ERR_CUDA;
}

extern "C" int bf_ragged_plan_destroy(bf_ragged_plan_t plan) {
    if (!plan) return -1;
    cudaGraphExecDestroy(plan->exec);
    cudaGraphDestroy(plan->graph);
    delete plan;
    return BF_SUCCESS;
}

extern "C" int bf_ragged_plan_info(bf_ragged_plan_t plan, int* out) {
    if (!plan) return -1;
    if (!out) return -2;
    out[0] = plan->p.nbig;
    out[1] = plan->p.nitems;
    out[2] = plan->blocks;
    out[3] = plan->threads;
    out[4] = (int)plan->smem;
    return BF_SUCCESS;
}

// ----------------------------------------------------------------------------- allocation-free entry point
// Some callers cannot allocate device memory when they solve: code running under a fixed
// memory budget (an embedded or real-time controller that sizes all memory at start-up and
// forbids allocation in its control loop, the setting the paper's routines are written for),
// and code that hands the library no workspace because another allocator owns the device.
// bf_ragged_potrf_potrs_noalloc serves them: the persistent kernel's queue lives in the
// file-scope array below, which every GPU that loads this library holds until the process
// exits, and the call allocates nothing (no cudaMalloc/cudaFree, no host heap).
#include <mutex>

#define BF_NOALLOC_ALIGN(x) (((x) + 255) / 256 * 256)

static constexpr size_t kNoallocCounter = 256;
static constexpr size_t kNoallocInts = BF_NOALLOC_ALIGN(sizeof(int) * (size_t)BF_RAGGED_NOALLOC_MAX);
static constexpr size_t kNoallocLongs = BF_NOALLOC_ALIGN(sizeof(long long) * (size_t)BF_RAGGED_NOALLOC_MAX);
static constexpr size_t kNoallocBytes = kNoallocCounter + 2 * kNoallocInts + 2 * kNoallocLongs;

static __device__ __align__(256) unsigned char g_ragged_noalloc_scratch[kNoallocBytes];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256];  // device address of the scratch array, per device ordinal
// host-side queue construction, reused by every call (guarded by g_noalloc_mu)
int h_order[BF_RAGGED_NOALLOC_MAX];
int h_n[BF_RAGGED_NOALLOC_MAX];
int h_orig[BF_RAGGED_NOALLOC_MAX];
long long h_offS[BF_RAGGED_NOALLOC_MAX];
long long h_offB[BF_RAGGED_NOALLOC_MAX];
}  // namespace

extern "C" int bf_ragged_potrf_potrs_noalloc(int batch, const int* n_host, int nrhs, double* S,
                                             const long long* offS_host, double* B, const long long* offB_host,
                                             int* info, int lane_max, int threads, bf_stream_t stream) {
    if (batch < 0) return -1;
    if (batch > 0 && !n_host) return -2;
    if (nrhs < 0 || nrhs > 64) return -3;
    if (batch > 0 && !S) return -4;
    if (batch > 0 && !offS_host) return -5;
    if (batch > 0 && nrhs > 0 && !B) return -6;
    if (batch > 0 && nrhs > 0 && !offB_host) return -7;
    if (lane_max < 0) return -9;
    if (threads != 64 && threads != 128 && threads != 256 && threads != 512) return -10;
    if (batch > BF_RAGGED_NOALLOC_MAX) return BF_ERR_NOALLOC_LIMIT;
    if (batch == 0) return BF_SUCCESS;
    int nmax = 0;
    for (int b = 0; b < batch; b++) {
        if (n_host[b] < 0) return -2;
        nmax = std::max(nmax, n_host[b]);
    }
    const size_t smem = bf::ragged_smem_bytes(nmax > lane_max ? nmax : 0, nrhs, threads);
    if (smem > 227 * 1024 || (nmax > lane_max && nmax > BF_BIG_NMAX)) return BF_ERR_NOT_SUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return BF_ERR_CUDA;
    // The queue goes to the device by copies from this file's host arrays, which the next call
    // overwrites: a captured copy would replay whatever queue the latest call left there.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) return BF_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return BF_ERR_NOT_SUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    // set-up, once per device, with that device current (the address stays valid for the life
    // of the device's context: after cudaDeviceReset it would be stale)
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_ragged_noalloc_scratch) != cudaSuccess || !ptr) return BF_ERR_CUDA;
        g_noalloc_ptr[dev] = ptr;
    }
    char* w = (char*)g_noalloc_ptr[dev];
    unsigned int* counter = (unsigned int*)w;
    int* dn = (int*)(w + kNoallocCounter);
    int* dorig = (int*)(w + kNoallocCounter + kNoallocInts);
    long long* doS = (long long*)(w + kNoallocCounter + 2 * kNoallocInts);
    long long* doB = (long long*)(w + kNoallocCounter + 2 * kNoallocInts + kNoallocLongs);
    // queue order: decreasing order n, ties by index (in place, no allocation)
    for (int i = 0; i < batch; i++) h_order[i] = i;
    std::sort(h_order, h_order + batch, [&](int a, int b) {
        return n_host[a] > n_host[b] || (n_host[a] == n_host[b] && a < b);
    });
    int nbig = 0;
    while (nbig < batch && n_host[h_order[nbig]] > lane_max) nbig++;
    for (int i = 0; i < batch; i++) {
        const int b = h_order[i];
        h_n[i] = n_host[b];
        h_orig[i] = b;
        h_offS[i] = offS_host[b];
        h_offB[i] = nrhs ? offB_host[b] : 0;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // pageable copies are staged before cudaMemcpyAsync returns, so the host arrays may be reused
    if (cudaMemcpyAsync(dn, h_n, sizeof(int) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dorig, h_orig, sizeof(int) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(doS, h_offS, sizeof(long long) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(doB, h_offB, sizeof(long long) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(counter, 0, sizeof(unsigned int), s) != cudaSuccess)  // the queue starts empty
        return BF_ERR_CUDA;
    bf::RaggedParams p;
    p.n = dn;
    p.offS = doS;
    p.offB = doB;
    p.orig = dorig;
    p.S = S;
    p.B = B;
    p.info = info;
    p.nrhs = nrhs;
    p.nbig = nbig;
    p.nprob = batch;
    p.nitems = nbig + (batch - nbig + threads - 1) / threads;
    p.counter = counter;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (smem + bf::kStaticSmemSlack > 48 * 1024 &&
        cudaFuncSetAttribute(bf::ragged_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return BF_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bf::ragged_persistent_kernel, threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return BF_ERR_CUDA;
    bf::ragged_persistent_kernel<<<sms * per_sm, threads, smem, s>>>(p);
    bf::count_launch();
    return cudaGetLastError() == cudaSuccess ? BF_SUCCESS : BF_ERR_CUDA;
}
