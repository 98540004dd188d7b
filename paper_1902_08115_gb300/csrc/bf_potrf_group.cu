// bf_potrf_group.cu -- dpotrf of small batches of small orders, element-parallel in shared
// memory (section 3.1 "dpotrf": the unblocked Cholesky recurrence, right-looking).
//
// One CTA factors a group of P problems at a time.  The group's lower triangles are copied into
// shared memory, problem-interleaved (slot e of problem p at S[e * PS + p]), and the right-looking
// recurrence runs column by column, every FP64 operation a unit (element, problem):
//
//   pivot   l_jj = sqrt(a_jj), r_j = 1 / l_jj                               (P units)
//   scale   l_ij = (a_ij - l_i,j-1 l_j,j-1) r_j     for i > j               (P (n-1-j) units)
//   update  a_ik -= l_ij l_kj                        for j+1 < k <= i        (P m(m-1)/2 units)
//
// (the update of column j+1 by column j is folded into its scale step of the next column).
// Why this shape on this GPU (measured with the library's FP64 probes): the SM's FP64 unit
// takes about one warp instruction per 16 cycles whatever the instruction's active lanes, and
// one warp issues at most one FP64 instruction per 64 cycles.  A batch too small to give every
// SM several warps of whole problems (one problem per lane needs ~20,000 problems) therefore
// leaves FP64 units idle in the lane form and wastes lanes in forms with a warp per problem.
// Here the units of a step fill the lanes of the CTA's warps whatever P is, and P can be any
// size (4096 problems: 27 per SM on 152 SMs, or 14 in each of two groups per SM).  Every FP64
// instruction but the pivots' does useful arithmetic; shared-memory traffic, index arithmetic
// and barriers issue beside the FP64 instructions.
//
// Element slots: columns in decreasing order, rows increasing inside a column, so that
// slot(i, k) = (n-1-k)(n-k)/2 + (i - k) and the trailing triangle of step j (columns > j) is
// the prefix of length m(m+1)/2, m = n-1-j: an update unit's own slot is its unit index.
//
// info follows LAPACK: the first column whose pivot is not positive (or NaN), 1-based, else 0.
// A failed problem keeps running on NaN; only its columns from the failing one on change,
// which LAPACK leaves unspecified.  info is written for every problem (no reset needed).
#include <atomic>

#include "bf_internal.h"

namespace bf {

__device__ __forceinline__ int group_slot(int n, int i, int k) { return (n - 1 - k) * (n - k) / 2 + (i - k); }

// Units u = tid, tid + NT, ... of a phase enumerate (a, b) = (u / P, u % P) without a division
// per unit: the per-thread start and the per-step increments are fixed for the kernel.
struct UnitStep {
    int a0, b0, da, db, P;
    __device__ __forceinline__ UnitStep(int tid, int NT, int P_) : P(P_) {
        a0 = tid / P_;
        b0 = tid - a0 * P_;
        da = NT / P_;
        db = NT - da * P_;
    }
    __device__ __forceinline__ void next(int& a, int& b) const {
        a += da;
        b += db;
        if (b >= P) {
            b -= P;
            a++;
        }
    }
};

// Shared memory: S (E slots x PS, PS = P rounded up to odd so that the copies' strided accesses
// spread over the banks), R (2 x P reciprocal pivots), T (E slot coordinates), F (P infos).
__host__ __device__ inline int group_stride(int P) { return P | 1; }

// Pivot of column j of problem p in slot c: info on the first non-positive (or NaN) pivot,
// l_jj = d / sqrt(d), and its reciprocal kept for the scale step.
__device__ __forceinline__ void group_pivot(double* S, double* R, int* F, int c, int PS, int p, int j, double d) {
    // d > 0 (not zero, negative or NaN) tested on the bits, which leaves the FP64 unit to the
    // arithmetic: positive finite or +inf is 0 < bits <= the bits of +inf
    const long long b = __double_as_longlong(d);
    if (!(b > 0 && b <= 0x7ff0000000000000ll) && F[p] == 0) F[p] = j + 1;
    const double rs = rsqrt(d);
    S[c * PS + p] = d * rs;
    R[p] = rs;
}

// Named barriers (id, thread count): a warp arrives without waiting, or waits for the count.
__device__ __forceinline__ void group_bar_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void group_bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Bulk update units [u, u1) of step j (stride NB, stepping state e, p carried across calls):
// a_ik -= l_ij l_kj, slot e of problem p.  Eight units in flight per thread: every load of a
// batch is issued before its first multiply-add, so a warp's FP64 instructions are not spaced
// out by shared-memory latency (the FP64 unit is shared by the SM's warps; each waits its turn).
template <int NB>
__device__ __forceinline__ void group_bulk(double* S, const int* T, int PS, int c0, const UnitStep& bs, int& u, int u1,
                                           int& e, int& p) {
    for (; u + 7 * NB < u1; u += 8 * NB) {
        int d[8], pi[8], pk[8];
#pragma unroll
        for (int x = 0; x < 8; x++) {
            const int ik = T[e], i = ik >> 16, k = ik & 0xffff;
            d[x] = e * PS + p;
            pi[x] = (c0 + i) * PS + p;
            pk[x] = (c0 + k) * PS + p;
            bs.next(e, p);
        }
        double a[8], li[8], lk[8];
#pragma unroll
        for (int x = 0; x < 8; x++) {
            a[x] = S[d[x]];
            li[x] = S[pi[x]];
            lk[x] = S[pk[x]];
        }
#pragma unroll
        for (int x = 0; x < 8; x++) S[d[x]] = fma(-li[x], lk[x], a[x]);
    }
    for (; u + 3 * NB < u1; u += 4 * NB) {
        int d[4], pi[4], pk[4];
#pragma unroll
        for (int x = 0; x < 4; x++) {
            const int ik = T[e], i = ik >> 16, k = ik & 0xffff;
            d[x] = e * PS + p;
            pi[x] = (c0 + i) * PS + p;
            pk[x] = (c0 + k) * PS + p;
            bs.next(e, p);
        }
        double a[4], li[4], lk[4];
#pragma unroll
        for (int x = 0; x < 4; x++) {
            a[x] = S[d[x]];
            li[x] = S[pi[x]];
            lk[x] = S[pk[x]];
        }
#pragma unroll
        for (int x = 0; x < 4; x++) S[d[x]] = fma(-li[x], lk[x], a[x]);
    }
    for (; u < u1; u += NB) {
        const int ik = T[e], i = ik >> 16, k = ik & 0xffff;
        double* sd = S + e * PS + p;
        *sd = fma(-S[(c0 + i) * PS + p], S[(c0 + k) * PS + p], *sd);
        bs.next(e, p);
    }
}

// Schedule: the serial chain of the recurrence (pivot, then the next column's first row, then
// the next pivot ...) is carried by warp 0 alone; warps 1.. carry the rest.  Invariant at the
// start of step j: columns < j final; column j has its pivot and row j+1; its rows j+2.. still
// lack the update by column j-1 and the scale; the columns > j are updated by columns < j.
//   warp 0      pivot of column j+1, then (after warps 1.. have row j+2 of column j) row j+2 of
//               column j+1
//   warps 1..   rows j+2.. of column j (update by column j-1, scale by r_j; row j+2 first, for
//               warp 0), a barrier among themselves, then the update of the columns > j+1 by
//               column j
// and one CTA barrier per step.  The reciprocal pivots of consecutive columns alternate between
// two arrays, since warp 0 writes r_j+1 while the others still scale by r_j.
template <int NW, bool UP>
__global__ void __launch_bounds__(32 * NW) dpotrf_group_kernel(int n, MatRef A, int lda, long long batch,
                                                              int* info, int P) {
    constexpr int NT = 32 * NW, NB = NT - 32;  // threads; bulk threads
    extern __shared__ double sm[];
    const int E = n * (n + 1) / 2;
    const int PS = group_stride(P);
    double* S = sm;
    double* R = S + (size_t)E * PS;
    int* T = reinterpret_cast<int*>(R + 2 * P);  // (i << 16) | k of every slot
    int* F = T + E;
    const int tid = threadIdx.x;
    const bool w0 = tid < 32;
    const int bt = tid - 32;  // rank among the bulk threads
    for (int e = tid; e < E; e += NT) {
        int t = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
        while ((t + 1) * (t + 2) / 2 <= e) t++;
        while (t * (t + 1) / 2 > e) t--;
        const int k = n - 1 - t, i = k + (e - t * (t + 1) / 2);
        T[e] = (i << 16) | k;
    }
    const UnitStep bs(w0 ? 0 : bt, NB, P);  // (slot or row, problem) units of the bulk threads
    const UnitStep ls(tid, NT, E);          // (problem, slot) units of the copies
    const long long groups = (batch + P - 1) / P;
    const int UC = P * E;
    for (long long g = blockIdx.x; g < groups; g += gridDim.x) {
        const long long q0 = g * P;
        const int np = (int)(batch - q0 < P ? batch - q0 : P);
        __syncthreads();  // the table is written / the previous group is stored
        // copy in: problem-major units, so that consecutive threads read consecutive rows, as
        // asynchronous copies straight into shared memory (all of a thread's in flight at once)
        {
            int p = ls.a0, e = ls.b0;
            for (int u = tid; u < UC; u += NT) {
                if (p < np) {
                    const int ik = T[e], i = ik >> 16, k = ik & 0xffff;
                    const double* a = A.ptr(q0 + p) + (UP ? k + (long long)i * lda : i + (long long)k * lda);
                    const unsigned sa = (unsigned)__cvta_generic_to_shared(S + e * PS + p);
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(a) : "memory");
                } else {
                    S[e * PS + p] = 0.0;
                }
                ls.next(p, e);
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
        }
        for (int p = tid; p < P; p += NT) F[p] = 0;
        __syncthreads();
        // column 0: pivot and row 1 (warp 0)
        const int c00 = group_slot(n, 0, 0);
        if (w0) {
            for (int p = tid; p < P; p += 32) {
                group_pivot(S, R, F, c00, PS, p, 0, S[c00 * PS + p]);
                if (n > 1) S[(c00 + 1) * PS + p] *= R[p];
            }
        }
        __syncthreads();
        for (int j = 0; j + 1 < n; j++) {
            const int m = n - 1 - j;
            const int c0 = group_slot(n, j, j) - j;  // l_xj in slot c0 + x
            const int es = (m - 1) * m / 2;         // slot of (j+1, j+1); column j+1 is es .. es+m-1
            const double* Rj = R + (j & 1) * P;     // reciprocal pivots of column j
            const bool row2 = j + 2 < n;            // column j has a row j+2
            const int wrow = (P + 31) / 32;         // warps 1 .. wrow compute row j+2 of column j
            if (w0) {
                // pivot of column j+1, then (once row j+2 of column j is in) its row j+2
                double* Rn = R + ((j + 1) & 1) * P;
                for (int p = tid; p < P; p += 32) {
                    const double l = S[(c0 + j + 1) * PS + p];
                    group_pivot(S, Rn, F, es, PS, p, j + 1, fma(-l, l, S[es * PS + p]));
                }
                if (row2) {
                    group_bar_sync(2, 32 * (1 + wrow));
                    for (int p = tid; p < P; p += 32) {
                        const int s = (es + 1) * PS + p;
                        S[s] = fma(-S[(c0 + j + 2) * PS + p], S[(c0 + j + 1) * PS + p], S[s]) * Rn[p];
                    }
                }
            } else {
                // rows j+2 .. of column j: the update by column j-1 (deferred from the previous
                // step) and the scale by r_j; row j+2 first, for warp 0
                const int cp0 = j > 0 ? group_slot(n, j - 1, j - 1) - (j - 1) : 0;  // l_x,j-1 in slot cp0 + x
                if (row2 && bt < 32 * wrow) {
                    if (bt < P) {
                        const int s = (c0 + j + 2) * PS + bt;
                        double v = S[s];
                        if (j > 0) v = fma(-S[(cp0 + j + 2) * PS + bt], S[(cp0 + j) * PS + bt], v);
                        S[s] = v * Rj[bt];
                    }
                    group_bar_arrive(2, 32 * (1 + wrow));
                }
                {
                    int r = bs.a0, q = bs.b0;
                    for (int v = bt; v < P * (m - 2); v += NB) {
                        const int i = j + 3 + r;
                        const int s = (c0 + i) * PS + q;
                        double a = S[s];
                        if (j > 0) a = fma(-S[(cp0 + i) * PS + q], S[(cp0 + j) * PS + q], a);
                        S[s] = a * Rj[q];
                        bs.next(r, q);
                    }
                }
                group_bar_sync(3, NB);
                // bulk update of the columns > j+1 (slots 0 .. es-1) by column j
                int e = bs.a0, p = bs.b0, u = bt;
                group_bulk<NB>(S, T, PS, c0, bs, u, P * es, e, p);
            }
            __syncthreads();
        }
        // copy out: the lower triangle (upper: its transpose) of each problem, and info
        {
            int p = ls.a0, e = ls.b0;
            for (int u = tid; u < UC; u += NT) {
                if (p < np) {
                    const int ik = T[e], i = ik >> 16, k = ik & 0xffff;
                    double* a = A.mptr(q0 + p);
                    (UP ? a[k + (long long)i * lda] : a[i + (long long)k * lda]) = S[e * PS + p];
                }
                ls.next(p, e);
            }
        }
        if (info)
            for (int p = tid; p < np; p += NT) info[q0 + p] = F[p];
    }
}

// Problems per group at most: row j+2 of a column is one unit per bulk thread (at least 128).
constexpr int kGroupMaxP = 128;

size_t potrf_group_smem(int n, int P) {
    const size_t E = (size_t)n * (n + 1) / 2;
    return E * group_stride(P) * sizeof(double) + 2 * (size_t)P * sizeof(double) + E * sizeof(int) +
           (size_t)P * sizeof(int);
}

// Problems per group: the batch spread over per_sm groups per SM, capped by shared memory.
int potrf_group_size(int n, long long batch, int per_sm) {
    long long P = (batch + kSMs * per_sm - 1) / (kSMs * per_sm);
    if (P < 1) P = 1;
    if (P > kGroupMaxP) P = kGroupMaxP;  // row j+2 of a column is one unit per bulk thread
    while (P > 1 && potrf_group_smem(n, (int)P) > kGroupSmemMax) P--;
    return (int)P;
}

// Problems per group from a model of the launch's time, for CTAs of `threads` threads using
// `regs` registers each on SMs with smem_sm bytes of shared memory (reserved_cta of it taken
// by every CTA).  With P problems per group, r CTAs resident per SM (shared memory,
// registers, threads) and W waves of 152 r CTAs, a wave costs the serial column chain once
// (the CTAs of an SM run their chains side by side) plus the update work of the problems on
// its busiest SM.  Counted in one problem's update work:
//   T(P) = W a ceil(P / 32) + P (r (W - 1) + c_last) + p CTAs_per_SM
// with c_last the CTAs on the busiest SM in the last wave, a = 9360 / n^2 (the chain's
// ~1,300 cycles per column against n^3/3 flops at ~2.4 per cycle per SM; warp 0 carries 32
// problems' chains per pass) and p = 922 / n^2 the pivot slots a group adds (8 FP64
// instructions per column whatever its P).  Measured on GB300 the model's choice matches the
// best of a sweep over P: n = 64 x 4,096 problems: P = 9, 788 GFLOP/s (13 problems per
// group, the shared-memory cap of two groups per SM: 583, its third wave 12 CTAs);
// n = 96 x 1,216: P = 4, 779 (5: 674); n = 32 x 12,288: P = 21, 754 (27: 666);
// n = 16 x 16,384: P = 54, 513 (36: 473).
int potrf_group_size_model(int n, long long batch, int threads, int regs, int smem_sm, int reserved_cta) {
    const double a = 9360.0 / ((double)n * n), piv = 922.0 / ((double)n * n);
    int bestP = 1;
    double bestT = -1.0;
    for (int P = 1; P <= kGroupMaxP; P++) {
        const size_t sm = potrf_group_smem(n, P);
        if (sm > kGroupSmemMax) break;
        long long r = (long long)smem_sm / ((long long)sm + reserved_cta);
        const long long r_reg = 65536 / ((long long)(regs > 0 ? regs : 1) * threads), r_thr = 2048 / threads;
        if (r_reg < r) r = r_reg;
        if (r_thr < r) r = r_thr;
        if (r > 32) r = 32;
        if (r < 1) break;
        const long long groups = (batch + P - 1) / P, slots = kSMs * r;
        const long long W = (groups + slots - 1) / slots;
        const long long rem = groups - slots * (W - 1), clast = (rem + kSMs - 1) / kSMs;
        const double T = W * a * (double)((P + 31) / 32) + P * (double)(r * (W - 1) + clast) +
                         piv * (double)((groups + kSMs - 1) / kSMs);
        if (bestT < 0.0 || T < bestT) {
            bestT = T;
            bestP = P;
        }
        if (groups == 1) break;  // larger groups only add empty slots
    }
    return bestP;
}

// Once per kernel instance (not on every call: attribute calls are host time that a small
// launch would wait for): the dynamic shared memory limit raised to the bound, and the
// registers per thread that the group-size model needs.
template <int NW, bool UP>
static cudaError_t group_prepare(int* regs) {
    static std::atomic<int> done{0};
    int d = done.load(std::memory_order_acquire);
    if (d) {
        *regs = d;
        return cudaSuccess;
    }
    cudaError_t e = cudaFuncSetAttribute(dpotrf_group_kernel<NW, UP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kGroupSmemMax);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, dpotrf_group_kernel<NW, UP>);
    if (e != cudaSuccess) return e;
    d = fa.numRegs > 0 ? fa.numRegs : 1;
    done.store(d, std::memory_order_release);
    *regs = d;
    return cudaSuccess;
}

// Shared memory per SM and per CTA reservation of the current device, once.
static void group_device_smem(int* smem_sm, int* reserved) {
    static std::atomic<int> s_sm{0}, s_res{-1};
    int a = s_sm.load(std::memory_order_acquire), b = s_res.load(std::memory_order_acquire);
    if (a == 0 || b < 0) {
        int dev = 0;
        a = 233472;  // GB300: 228 KB per SM, 1 KB reserved per CTA
        b = 1024;
        if (cudaGetDevice(&dev) == cudaSuccess) {
            int v = 0;
            if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess && v > 0) a = v;
            if (cudaDeviceGetAttribute(&v, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess && v >= 0) b = v;
        }
        s_sm.store(a, std::memory_order_release);
        s_res.store(b, std::memory_order_release);
    }
    *smem_sm = a;
    *reserved = b;
}

template <int NW>
static cudaError_t launch_group(int n, MatRef A, int lda, long long batch, int* info, cudaStream_t s, int upper,
                                int per_sm) {
    int regs = 0;
    cudaError_t e = upper ? group_prepare<NW, true>(&regs) : group_prepare<NW, false>(&regs);
    if (e != cudaSuccess) return e;
    int P;
    if (per_sm > 0) {
        P = potrf_group_size(n, batch, per_sm);
    } else {
        int smem_sm, reserved;
        group_device_smem(&smem_sm, &reserved);
        P = potrf_group_size_model(n, batch, 32 * NW, regs, smem_sm, reserved);
    }
    const size_t smem = potrf_group_smem(n, P);
    if (smem > kGroupSmemMax) return cudaErrorInvalidValue;
    const long long groups = (batch + P - 1) / P;
    const long long cap = kSMs * 8;
    const unsigned blocks = (unsigned)(groups < cap ? groups : cap);
    if (upper) {
        dpotrf_group_kernel<NW, true><<<blocks, 32 * NW, smem, s>>>(n, A, lda, batch, info, P);
    } else {
        dpotrf_group_kernel<NW, false><<<blocks, 32 * NW, smem, s>>>(n, A, lda, batch, info, P);
    }
    count_launch();
    return cudaGetLastError();
}

// threads: 256, 384 or 512 per CTA; per_sm: groups per SM that the batch is spread over (1..4),
// or 0: the group size from the time model (potrf_group_size_model)
cudaError_t launch_dpotrf_group(int n, MatRef A, int lda, long long batch, int* info, cudaStream_t s, int upper,
                                int threads, int per_sm) {
    if (batch == 0 || n == 0) return cudaSuccess;
    if (per_sm < 0) per_sm = 0;
    if (per_sm > 4) per_sm = 4;
    if (threads == 384) return launch_group<12>(n, A, lda, batch, info, s, upper, per_sm);
    if (threads == 512) return launch_group<16>(n, A, lda, batch, info, s, upper, per_sm);
    return launch_group<8>(n, A, lda, batch, info, s, upper, per_sm);
}

}  // namespace bf
