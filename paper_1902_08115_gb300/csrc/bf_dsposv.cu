// bf_dsposv.cu -- batched mixed-precision SPD solve: binary32 Cholesky factor,
// binary64 iterative refinement (the interface is LAPACK's dsposv, including
// its workspace).
//
// The factorisation and solves are the paper's dpotrf/dtrsm (section 3.1)
// carried out in binary32; refinement recovers binary64 accuracy.  One CTA
// (128 threads) per problem, the binary32 factor in shared memory (columns in
// 16-byte-aligned groups of four rows):
//   1. A's lower triangle is rounded to binary32 and factored A32 = L32 L32^T,
//      right-looking with 8-column panels: the panel by one warp, in registers
//      with shuffles (each pivot tested for positivity; its binary64 square
//      root rounded to binary32 is the correctly rounded binary32 one), the
//      trailing update by all threads on 4x4 tiles of 16-byte pieces -- two
//      barriers per panel.
//   2. x = L32^{-T} L32^{-1} b (binary32 substitutions by one warp, the vector
//      in registers, x kept in binary64); repeat: r = b - A x in binary64 (A symmetric from its lower
//      triangle, read from global memory); stop when the normwise backward
//      error eta = ||r||_inf / (||A||_inf ||x||_inf + ||b||_inf) <= tol;
//      d = L32^{-T} L32^{-1} r (binary32); x = x + d in binary64.
//   3. If the binary32 factorisation fails (a pivot <= 0, NaN, or an entry
//      outside the binary32 range) or `itmax` steps do not reach tol, the
//      problem is factored and solved in binary64 in its workspace slice
//      (iter = -1), as LAPACK's dsposv does.
// The warp that runs the serial phases is rotated by problem index, so the
// serial phases of co-resident CTAs spread over the SM's four sub-partitions.
// ||A||_inf is accumulated in binary32 from the rounded entries and scaled by
// (1 - 2(n+2) 2^-24): a lower bound of the binary64 norm, so the stopping
// test never under-estimates eta.  binary64 -> binary32
// conversions of matrix entries are integer operations (round to nearest
// even, binary32 subnormals included, as the IEEE conversion): FP64
// instructions run at 1/64 of the binary32 rate on this GPU.
#include "bf_internal.h"
#include "../../include/bfgpu.h"

namespace bf {

// ---------------------------------------------------------------- binary64 -> binary32 by integer operations
__device__ __noinline__ float f64_to_f32_rn(double a) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(a);
    const unsigned int sign = (unsigned int)(u >> 63) << 31;
    const int e = (int)((u >> 52) & 0x7FF);
    const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
    if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));  // inf / NaN
    int E = e - 1023 + 127;
    if (e == 0) return __uint_as_float(sign);  // binary64 zero or subnormal: below half the binary32 minimum
    if (E <= 0) {
        // below the binary32 normal range: round sig 2^(e-1075) to a multiple of 2^-149 (a binary32
        // subnormal, or the smallest normal when it rounds up to 2^-126), ties to even
        const unsigned long long sig = m | (1ull << 52);
        const int sh = 926 - e;  // 1075 - 149 - e, at least 30 here
        if (sh > 54) return __uint_as_float(sign);
        unsigned long long q = sig >> sh;
        const unsigned long long rem = sig & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (q & 1ull))) q++;
        return __uint_as_float(sign | (unsigned int)q);
    }
    unsigned int mant = (unsigned int)(m >> 29);
    const unsigned int rem = (unsigned int)(m & 0x1FFFFFFFull);
    if (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) {
        mant++;
        if (mant == 0x800000u) {
            mant = 0;
            E++;
        }
    }
    if (E >= 255) return __uint_as_float(sign | 0x7F800000u);
    return __uint_as_float(sign | ((unsigned int)E << 23) | mant);
}

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
    unsigned char* work;  // per problem: `wper` bytes for the binary64 fallback factor
    long long wper;
};

// ---------------------------------------------------------------- one CTA per problem
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

// block-wide max of non-negative values given as order-preserving bit patterns
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

// packed lower triangle by columns (the binary64 fallback's factor in the workspace)
__device__ __forceinline__ int pk(int i, int j, int n) { return j * n - (j * (j - 1)) / 2 + (i - j); }

// Storage of the binary32 factor in shared memory: column j holds rows 4 floor(j/4) .. n4 - 1
// (n4 = n rounded up to a multiple of 4), the columns one after another, so that
// L(i, j) = L[cb(j, n4) + i] and four rows starting at a multiple of 4 are one aligned 16-byte
// piece.  The rows above the diagonal inside a column's group of four, and the rows n .. n4 - 1,
// are padding.  n4 * n4 / 2 + 2 n4 floats in all.
__device__ __forceinline__ int cb(int j, int n4) {
    const int g = j >> 2, r = j & 3;
    return 4 * n4 * g - 8 * g * (g - 1) + r * (n4 - 4 * g) - 4 * g;
}

// w <- L^{-T} L^{-1} w with the binary32 factor in shared memory, by one warp with w in
// registers: lane l holds w_i for i = l, l + 32, ...; each step broadcasts the solved entry
// from its lane and every lane updates its own entries (a column of L for the forward solve,
// contiguous in storage; a row for the backward one).  The steps are unrolled two at a time:
// the loads of L and of the reciprocal pivots, which do not depend on w, are then issued a step
// ahead (16,384 x n = 128: 3.64 -> 3.52 ms; unrolled 4, 8 or 32 deep the kernel measured
// slower, 3.71 / 3.89 / 4.70 ms, its code outgrowing the instruction cache).  The step order
// and every operation are those of the plain loop, so the results are the same bits.
template <int NR>
__device__ __noinline__ void solve32_warp(const float* L, const float* rinv, float* w, int n) {
    const int lane = threadIdx.x & 31;
    const int n4 = (n + 3) & ~3;
    float x[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) x[r] = (lane + 32 * r < n) ? w[lane + 32 * r] : 0.0f;
#pragma unroll
    for (int s = 0; s < NR; s++) {
        if (32 * s >= n) break;
#pragma unroll 2
        for (int lj = 0; lj < 32; lj++) {
            const int j = 32 * s + lj;
            if (j >= n) break;
            const float* col = L + cb(j, n4);  // col[i] = L(i, j)
            const float yj = __shfl_sync(0xffffffffu, x[s], lj) * rinv[j];
            if (lane == lj) x[s] = yj;
#pragma unroll
            for (int s2 = s; s2 < NR; s2++) {
                const int i = lane + 32 * s2;
                if ((s2 > s || lane > lj) && i < n) x[s2] = fmaf(-col[i], yj, x[s2]);
            }
        }
    }
    int base[NR];  // L(j, i) = L[base + j] for this lane's rows i
#pragma unroll
    for (int r = 0; r < NR; r++) base[r] = cb(imin(lane + 32 * r, n - 1), n4);
#pragma unroll
    for (int s = NR - 1; s >= 0; s--) {
        if (32 * s >= n) continue;
#pragma unroll 2
        for (int lj = 31; lj >= 0; lj--) {
            const int j = 32 * s + lj;
            if (j >= n) continue;
            const float xj = __shfl_sync(0xffffffffu, x[s], lj) * rinv[j];
            if (lane == lj) x[s] = xj;
#pragma unroll
            for (int s2 = 0; s2 <= s; s2++) {
                if (s2 < s || lane < lj) x[s2] = fmaf(-L[base[s2] + j], xj, x[s2]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < NR; r++)
        if (lane + 32 * r < n) w[lane + 32 * r] = x[r];
}

// The panel J..J+nb (nb <= 8) of the binary32 factor, factored by one warp with the panel in
// registers: lane l holds rows J + l + 32 r.  Per column j = J + c: the pivot d (row j: lane c)
// is broadcast and tested; l_jj = sqrt(d) rounded to binary32, which equals the binary64 square
// root rounded to binary32 (double rounding of a square root is innocuous when the wider format
// has at least 2p + 2 significand bits: Figueroa, 1995; 53 >= 2 * 24 + 2); the column below is
// scaled by 1 / l_jj, and the panel's later columns are updated with the scaled multipliers.
// The code is straight-line (a failed or absent column continues with d = 1 and is reported),
// so that the shuffles of the next multipliers are issued while the pivot is being rooted:
// lane c2's scaled multiplier is its unscaled value times 1 / l_jj, formed here from a copy
// fetched ahead -- the same product, bit for bit.  1 / l_jj comes from the hardware's
// reciprocal square root of d refined by one Newton step y (3/2 - d y^2 / 2) (~1 ulp; the
// refinement in binary64 removes the factor's rounding, whatever it is).  Returns 0, or the
// 1-based column whose pivot is not positive (or not finite).
template <int NR>
__device__ int panel32_warp(float* L, float* rinv, int n, int J, int nb) {
    const int lane = threadIdx.x & 31;
    const int n4 = (n + 3) & ~3;
    float pnl[NR][8];
#pragma unroll
    for (int r = 0; r < NR; r++)
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const int i = J + lane + 32 * r;
            pnl[r][c] = (c < nb && i < n && i >= J + c) ? L[cb(J + c, n4) + i] : 0.0f;
        }
    int fail = 0;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int j = J + c;
        float u[8];  // unscaled L(J + c2, j), c2 > c
#pragma unroll
        for (int c2 = c + 1; c2 < 8; c2++) u[c2] = __shfl_sync(0xffffffffu, pnl[0][c], c2);
        float d = __shfl_sync(0xffffffffu, pnl[0][c], c);  // the same value in every lane
        const bool bad = !(d > 0.0f) || d == INFINITY;
        if (c < nb && bad && fail == 0) fail = j + 1;
        if (c >= nb || bad) d = 1.0f;
        const float y = rsqrtf(d);
        const float t = 0.5f * d * y;
        const float ri = fmaf(y, fmaf(-t, y, 0.5f), y);
        const float ljj = __fsqrt_rn(d);
        // unpredicated: entries on and above the diagonal and rows >= n are never stored
        // back, rows >= n hold zeros, and every value read below comes from a row > j
#pragma unroll
        for (int r = 0; r < NR; r++) pnl[r][c] *= ri;
        if (lane == c) pnl[0][c] = ljj;
        if (lane == 0 && c < nb) rinv[j] = ri;
#pragma unroll
        for (int c2 = c + 1; c2 < 8; c2++) {
            const float lk = u[c2] * ri;  // L(J + c2, j)
#pragma unroll
            for (int r = 0; r < NR; r++) pnl[r][c2] = fmaf(-pnl[r][c], lk, pnl[r][c2]);
        }
    }
#pragma unroll
    for (int r = 0; r < NR; r++)
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const int i = J + lane + 32 * r;
            if (c < nb && i < n && i >= J + c) L[cb(J + c, n4) + i] = pnl[r][c];
        }
    return fail;
}

static size_t factor_floats(int n) {
    const size_t n4 = (size_t)((n + 3) & ~3);
    return n4 * n4 / 2 + 2 * n4;
}

static size_t refine_smem_bytes(int n) {
    // factor | reciprocal pivots | w (binary32) | x, r (binary64) | scratch
    size_t f = (factor_floats(n) + (size_t)n + (size_t)n) * sizeof(float);
    f = (f + 15) / 16 * 16;
    return f + 2 * (size_t)n * sizeof(double) + 32 * sizeof(double);
}

// NR: rows per lane in the warp-register phases (n <= 32 NR); 4 keeps the panel in registers
template <int NR>
__global__ void __launch_bounds__(128, 6) dsposv_kernel(SposvParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const long long q = blockIdx.x;
    if (q >= p.batch) return;
    const int n = p.n;
    const int tid = threadIdx.x, T = blockDim.x, warp = tid >> 5, lane = tid & 31;
    const int sw = (int)(q % (T >> 5));  // the warp that runs the serial phases
    float* L = reinterpret_cast<float*>(smem_raw);
    const int n4 = (n + 3) & ~3;
    const int nf = n4 * n4 / 2 + 2 * n4;  // factor_floats(n)
    float* rinv = L + nf;
    float* wv = rinv + n;
    size_t off = ((size_t)nf + 2 * (size_t)n) * sizeof(float);
    off = (off + 15) / 16 * 16;
    double* xv = reinterpret_cast<double*>(smem_raw + off);
    double* rv = xv + n;
    unsigned long long* scratch = reinterpret_cast<unsigned long long*>(rv + n);
    __shared__ int s_done;

    const double* A = p.A.ptr(q);
    const double* B = p.B.ptr(q);
    double* X = p.X.mptr(q);
    unsigned char* wbytes = p.work + q * p.wper;

    // ---- 1. round the lower triangle to binary32: warp w takes columns w, w + 4, ...; its
    //         lanes read consecutive rows (coalesced) and write the column's whole storage,
    //         padding as zeros ----
    // Four columns per step, every load unconditional (rows clamped into j .. n - 1): all 4 NR
    // loads are in flight before the first conversion.
    const int nw = T >> 5;
    for (int j0 = warp; j0 < n; j0 += 4 * nw) {
        double v[4][NR];
#pragma unroll
        for (int h = 0; h < 4; h++) {
            const int j = imin(j0 + h * nw, n - 1);
            const double* a = A + (long long)j * p.lda;
#pragma unroll
            for (int r = 0; r < NR; r++) v[h][r] = a[imin(imax(4 * (j >> 2) + lane + 32 * r, j), n - 1)];
        }
#pragma unroll
        for (int h = 0; h < 4; h++) {
            const int j = j0 + h * nw;
            if (j >= n) continue;
            float* Lc = L + cb(j, n4);  // Lc[i] = L(i, j)
#pragma unroll
            for (int r = 0; r < NR; r++) {
                const int i = 4 * (j >> 2) + lane + 32 * r;
                if (i < n4) Lc[i] = (i >= j && i < n) ? f64_to_f32_rn(v[h][r]) : 0.0f;
            }
        }
    }
    if (tid == 0) s_done = 0;
    __syncthreads();
    // ||A||_inf of the symmetric matrix from the rounded lower triangle.  Each rounded entry
    // is at most (1 + 2^-24) times the binary64 one and a binary32 sum of n terms, in any
    // order, is accurate to (n + 1) 2^-24, so the scaled result is a lower bound of the
    // binary64 norm.  Row i: L(i, 0..i-1) along its row, then L(i..n-1, i) down its column.
    unsigned long long an = 0;
    for (int i = tid; i < n; i += T) {
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll 4
        for (int j = 0; j < i; j++) s0 += fabsf(L[cb(j, n4) + i]);
        const int off = cb(i, n4) + i;
        int k = 0;
        for (; k + 3 < n - i; k += 4) {
            s1 += fabsf(L[off + k]);
            s2 += fabsf(L[off + k + 1]);
            s3 += fabsf(L[off + k + 2]);
            s0 += fabsf(L[off + k + 3]);
        }
        for (; k < n - i; k++) s1 += fabsf(L[off + k]);
        const unsigned long long b = (unsigned long long)__float_as_uint((s0 + s1) + (s2 + s3));
        an = b > an ? b : an;
    }
    an = block_max_u64(an, scratch);
    const double anorm =
        (double)__uint_as_float((unsigned int)an) * (1.0 - 2.0 * (n + 2) * 5.9604644775390625e-08);

    // ---- 2. binary32 Cholesky, right-looking, 8-column panels ----
    for (int J = 0; J < n; J += 8) {
        const int nb = imin(8, n - J);
        if (warp == sw) {
            const int f = panel32_warp<NR>(L, rinv, n, J, nb);
            if (f && lane == 0) s_done = f;
        }
        __syncthreads();
        if (s_done) break;
        const int R = J + nb, m = n - R;
        if (m > 0) {
            const int tb = (m + 3) / 4;
            const int ntile = tb * (tb + 1) / 2;
            for (int t = tid; t < ntile; t += T) {
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
#pragma unroll
                for (int c = 0; c < 8; c++) {  // nb == 8 whenever a trailing matrix remains
                    // rows i0.., k0.. (multiples of 4, below the panel) as aligned 16-byte pieces;
                    // the zero padding rows n .. n4 - 1 only reach discarded tile entries
                    const float* col = L + cb(J + c, n4);
                    const float4 l4 = *reinterpret_cast<const float4*>(col + i0);
                    const float4 k4 = *reinterpret_cast<const float4*>(col + k0);
                    const float li[4] = {l4.x, l4.y, l4.z, l4.w}, lk[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
                    for (int a = 0; a < 4; a++)
#pragma unroll
                        for (int b = 0; b < 4; b++) acc[a][b] = fmaf(li[a], lk[b], acc[a][b]);
                }
                // rows i0 .. i0 + 3 of columns k0 .. k0 + 3, whole pieces: on a diagonal tile the
                // entries above the diagonal are padding, and padding rows receive zeros
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    const int k = k0 + b;
                    if (k >= n) continue;
                    float4* cp = reinterpret_cast<float4*>(L + cb(k, n4) + i0);
                    float4 v = *cp;
                    v.x -= acc[0][b];
                    v.y -= acc[1][b];
                    v.z -= acc[2][b];
                    v.w -= acc[3][b];
                    *cp = v;
                }
            }
        }
        __syncthreads();
    }
    bool fallback = s_done != 0;
    int iters = 0;

    // ---- 3. solve and refine every right-hand side ----
    for (int c = 0; c < p.nrhs && !fallback; c++) {
        const double* b = B + (long long)c * p.ldb;
        unsigned long long bn = 0;
        for (int i = tid; i < n; i += T) {
            const double bi = b[i];
            bn = absbits(bi) > bn ? absbits(bi) : bn;
            wv[i] = f64_to_f32_rn(bi);
        }
        bn = block_max_u64(bn, scratch);
        const double bnorm = __longlong_as_double((long long)bn);
        if (warp == sw) solve32_warp<NR>(L, rinv, wv, n);
        __syncthreads();
        for (int i = tid; i < n; i += T) xv[i] = (double)wv[i];
        __syncthreads();
        int it = 0;
        bool done = false;
        for (;;) {
            unsigned long long rn = 0, xn = 0;
            for (int i = tid; i < n; i += T) {
                // row i of the symmetric A: A(i, 0..i-1) along row i of the lower triangle
                // (consecutive threads, consecutive rows: coalesced), then A(i..n-1, i) down
                // column i (contiguous for the thread: 16-byte loads); four partial sums
                double s0 = b[i], s1 = 0.0, s2 = 0.0, s3 = 0.0;
                const double* ai = A + i;
                int j = 0;
                for (; j + 3 < i; j += 4) {
                    s0 = fma(-ai[(long long)j * p.lda], xv[j], s0);
                    s1 = fma(-ai[(long long)(j + 1) * p.lda], xv[j + 1], s1);
                    s2 = fma(-ai[(long long)(j + 2) * p.lda], xv[j + 2], s2);
                    s3 = fma(-ai[(long long)(j + 3) * p.lda], xv[j + 3], s3);
                }
                for (; j < i; j++) s0 = fma(-ai[(long long)j * p.lda], xv[j], s0);
                const double* ci = A + (long long)i * p.lda;
                int k = i;
                if ((reinterpret_cast<uintptr_t>(ci + k) & 15u) != 0) {
                    s1 = fma(-ci[k], xv[k], s1);
                    k++;
                }
                for (; k + 3 < n; k += 4) {
                    const double2 u = ldg2(ci + k), v = ldg2(ci + k + 2);
                    s0 = fma(-u.x, xv[k], s0);
                    s1 = fma(-u.y, xv[k + 1], s1);
                    s2 = fma(-v.x, xv[k + 2], s2);
                    s3 = fma(-v.y, xv[k + 3], s3);
                }
                for (; k < n; k++) s2 = fma(-ci[k], xv[k], s2);
                const double s = (s0 + s1) + (s2 + s3);
                rv[i] = s;
                rn = absbits(s) > rn ? absbits(s) : rn;
                xn = absbits(xv[i]) > xn ? absbits(xv[i]) : xn;
            }
            rn = block_max_u64(rn, scratch);
            __syncthreads();
            xn = block_max_u64(xn, scratch);
            const double rnorm = __longlong_as_double((long long)rn);
            const double xnorm = __longlong_as_double((long long)xn);
            if (rnorm <= p.tol * (anorm * xnorm + bnorm)) {
                done = true;
                break;
            }
            if (it == p.itmax) break;
            for (int i = tid; i < n; i += T) wv[i] = (float)rv[i];
            __syncthreads();
            if (warp == sw) solve32_warp<NR>(L, rinv, wv, n);
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

    // ---- binary64 fallback: factor (packed lower, in this problem's workspace) and solve ----
    __syncthreads();
    double* Lp = reinterpret_cast<double*>(wbytes);
    for (int e = tid; e < n * n; e += T) {
        const int j = e / n, i = e - j * n;
        if (i >= j) Lp[pk(i, j, n)] = A[i + (long long)j * p.lda];
    }
    if (tid == 0) s_done = 0;
    __syncthreads();
    for (int j = 0; j < n; j++) {
        const double d = Lp[pk(j, j, n)];
        if (!(d > 0.0)) {
            if (tid == 0) s_done = j + 1;
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
    const int finfo = s_done;
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

// workspace layout: per problem the binary64 packed lower triangle of the fallback, 256-byte aligned
static long long sposv_wper(int n) {
    const long long f64 = (long long)n * (n + 1) / 2 * (long long)sizeof(double);
    return (f64 + 255) / 256 * 256;
}

size_t dsposv_workspace_bytes(int n, long long batch) {
    if (n <= 0 || batch <= 0) return 0;
    return (size_t)(sposv_wper(n) * batch);
}

cudaError_t launch_dsposv(int n, int nrhs, MatRef A, int lda, MatRef B, int ldb, MatRef X, int ldx, int* iter,
                          int* info, double tol, int itmax, void* work, long long batch, cudaStream_t s) {
    if (batch == 0 || n == 0 || nrhs == 0) return cudaSuccess;
    SposvParams p;
    p.n = n; p.nrhs = nrhs; p.A = A; p.lda = lda; p.B = B; p.ldb = ldb; p.X = X; p.ldx = ldx;
    p.iter = iter; p.info = info; p.tol = tol; p.itmax = itmax; p.batch = batch;
    p.wper = sposv_wper(n);
    p.work = reinterpret_cast<unsigned char*>(work);
    const size_t smem = refine_smem_bytes(n);
    auto kfn = n <= 128 ? dsposv_kernel<4> : dsposv_kernel<BF_DSPOSV_NMAX / 32>;
    if (smem + kStaticSmemSlack > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kfn<<<(unsigned)batch, 128, smem, s>>>(p);
    count_launch();
    return cudaGetLastError();
}

}  // namespace bf

extern "C" size_t bf_dsposv_workspace_bytes(int n, int batch) { return bf::dsposv_workspace_bytes(n, batch); }

extern "C" int bf_dsposv_strided_batched(char uplo, int n, int nrhs, const double* A, int lda, long long strideA,
                                         const double* B, int ldb, long long strideB, double* X, int ldx,
                                         long long strideX, int* iter, int* info, double tol, int itmax,
                                         void* work, size_t work_bytes, int batch, bf_stream_t stream) {
    const bool lo = (uplo == 'L' || uplo == 'l'), up = (uplo == 'U' || uplo == 'u');
    if (!(lo || up)) return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (lda < (n > 1 ? n : 1)) return -5;
    if (strideA < 0) return -6;
    if (ldb < (n > 1 ? n : 1)) return -8;
    if (ldx < (n > 1 ? n : 1)) return -11;
    if (batch < 0) return -19;
    if (batch > 1 && strideX < (long long)ldx * nrhs) return -12;
    if (!(tol >= 0.0)) return -15;
    if (itmax < 0) return -16;
    const bool work_needed = n > 0 && nrhs > 0 && batch > 0;
    if (work_needed && !A) return -4;
    if (work_needed && !B) return -7;
    if (work_needed && !X) return -10;
    if (work_needed && work_bytes < bf::dsposv_workspace_bytes(n, batch)) return -18;
    if (work_needed && (!work || (reinterpret_cast<unsigned long long>(work) & 255ull))) return -17;
    if (up) return BF_ERR_NOT_SUPPORTED;
    if (n > BF_DSPOSV_NMAX) return BF_ERR_NOT_SUPPORTED;
    if (!work_needed) return 0;
    cudaError_t e = bf::launch_dsposv(n, nrhs, bf::mat_strided(A, strideA), lda, bf::mat_strided(B, strideB), ldb,
                                      bf::mat_strided(X, strideX), ldx, iter, info, tol, itmax, work, batch,
                                      (cudaStream_t)stream);
    return e == cudaSuccess ? BF_SUCCESS : BF_ERR_CUDA;
}
