// bf_dgemm.cu -- batched FP64 dgemm, C <= alpha op(A) op(B) + beta C (section 2.1).
//
// One thread computes one MR x NR register tile of C (the paper's kernel
// "size" m_r x n_r, section 3.2.1).  A CTA covers a TM x TN super-tile of P
// problems; thread (ri, rj) of a problem owns rows i0 + ri + GR*s (s < MR) and
// columns j0 + rj + GC*u (u < NR), GR = TM/MR, GC = TN/NR, so consecutive
// lanes touch consecutive rows.
//
// Two ways of feeding the k-loop, the two ends of the paper's algorithmic
// variants (section 2.2, table 1):
//   DIRECT (variant 'D'): op(A) and op(B) are read natively, column-major,
//     from global memory (through L1); no packing, no buffer.  The 'T' forms
//     read A across columns, the analogue of the paper's non-vectorisable
//     tn/tt direct kernels.
//   PACKED (variants 'B'/'C'): the CTA copies k-slices of op(A) and op(B)
//     into shared memory in a k-major panel layout, transposing while packing
//     so that the inner kernel is always the same (the paper's "transpose
//     while packing" rule, sections 2.2 and 3.2.1).
//
// The `tri` mask restricts stores to one triangle of C: TRI_LOWER (i >= j, the
// dsyrk-style trailing update of the blocked Cholesky, section 3.1
// "dsyrk"/"dpotrf"), TRI_UPPER (i <= j), TRI_SLOWER (i > j), TRI_SUPPER
// (i < j) -- the last ones for the triangular adjoints of the backward pass.
#include "bf_internal.h"

namespace bf {

template <int MR, int NR, bool TA, bool TB, bool PACKED, bool NEG>
__global__ void __launch_bounds__(512)
dgemm_tile_kernel(GemmParams p) {
    extern __shared__ double smem[];
    const int GR = p.TM / MR;
    const int GC = p.TN / NR;
    const int tpp = GR * GC;
    const int nst = p.tilesM * p.tilesN;
    const long long b = blockIdx.x;
    const int st = (int)(b % nst);
    const long long g = b / nst;
    const int i0 = (st % p.tilesM) * p.TM;
    const int j0 = (st / p.tilesM) * p.TN;

    // super-tiles with no element in the stored triangle
    if ((p.lower == TRI_LOWER && i0 + p.TM - 1 < j0) || (p.lower == TRI_SLOWER && i0 + p.TM - 1 <= j0) ||
        (p.lower == TRI_UPPER && i0 > j0 + p.TN - 1) || (p.lower == TRI_SUPPER && i0 >= j0 + p.TN - 1))
        return;

    const int t = threadIdx.x;
    const int ql = t / tpp;
    const int r = t - ql * tpp;
    const int ri = r % GR;
    const int rj = r / GR;
    const long long q = g * p.P + ql;
    bool valid = (ql < p.P) && (q < p.batch);
    if (valid && p.skip && p.skip[q] != 0) valid = false;

    const double* A = valid ? p.A.ptr(q) : nullptr;
    const double* B = valid ? p.B.ptr(q) : nullptr;
    double* C = valid ? p.C.mptr(q) : nullptr;

    int rows[MR], cols[NR];
#pragma unroll
    for (int s = 0; s < MR; s++) rows[s] = i0 + ri + GR * s;
#pragma unroll
    for (int u = 0; u < NR; u++) cols[u] = j0 + rj + GC * u;
    // clamped indices keep every load in bounds; out-of-range results are not stored
    int rc[MR], cc[NR];
#pragma unroll
    for (int s = 0; s < MR; s++) rc[s] = imin(rows[s], p.m - 1);
#pragma unroll
    for (int u = 0; u < NR; u++) cc[u] = imin(cols[u], p.n - 1);

    double acc[MR][NR];
    if (valid && (p.mode == ACC_C || p.mode == ACC_BC)) {
#pragma unroll
        for (int s = 0; s < MR; s++)
#pragma unroll
            for (int u = 0; u < NR; u++) acc[s][u] = C[rc[s] + (long long)cc[u] * p.ldc];
        if (p.mode == ACC_BC) {
#pragma unroll
            for (int s = 0; s < MR; s++)
#pragma unroll
                for (int u = 0; u < NR; u++) acc[s][u] *= p.beta;
        }
    } else {
#pragma unroll
        for (int s = 0; s < MR; s++)
#pragma unroll
            for (int u = 0; u < NR; u++) acc[s][u] = 0.0;
    }

    if (PACKED) {
        const int sAq = p.KC * p.TM + 1;  // per-problem stride (odd: staggers banks across problems)
        const int sBq = p.KC * p.TN + 1;
        double* sA = smem;
        double* sB = smem + (size_t)p.P * sAq;
        const int T = blockDim.x;
        for (int k0 = 0; k0 < p.k; k0 += p.KC) {
            const int kc = imin(p.KC, p.k - k0);
            // ---- pack op(A)(i0:i0+TM, k0:k0+kc) of every problem, k-major ----
            // Each thread moves two elements that are consecutive in memory (along i for A, along
            // p for A^T): one 16-byte load when the pair is in range and 16-byte aligned (even
            // leading dimension, aligned base), else single words.  Consecutive threads take
            // consecutive pairs: the warp reads 512 contiguous bytes.
            {
                const int ext = TA ? kc : p.TM;       // the contiguous extent
                const int hp = (ext + 1) >> 1;        // pairs along it
                const int np2 = p.P * hp * (TA ? p.TM : kc);
                for (int e = t; e < np2; e += T) {
                    const int h = e % hp;
                    const int rest = e / hp;
                    int qq, pp, ii;
                    if (!TA) {  // pair (ii, ii+1) in column k0 + pp
                        ii = 2 * h;
                        pp = rest % kc;
                        qq = rest / kc;
                    } else {  // pair (pp, pp+1) of row i0 + ii
                        pp = 2 * h;
                        ii = rest % p.TM;
                        qq = rest / p.TM;
                    }
                    const long long qg = g * p.P + qq;
                    double v0 = 0.0, v1 = 0.0;
                    const int gi = i0 + ii;
                    // validity of the first and second element of the pair
                    const bool in0 = qg < p.batch && gi < p.m && (TA ? pp < kc : true);
                    const bool in1 = qg < p.batch && (TA ? (gi < p.m && pp + 1 < kc) : (gi + 1 < p.m && ii + 1 < p.TM));
                    if (in0) {
                        const double* Aq = p.A.ptr(qg);
                        const double* src = TA ? Aq + (k0 + pp) + (long long)gi * p.lda
                                               : Aq + gi + (long long)(k0 + pp) * p.lda;
                        if (in1 && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
                            const double2 w = ldg2(src);
                            v0 = w.x;
                            v1 = w.y;
                        } else {
                            v0 = ldg(src);
                            if (in1) v1 = ldg(src + 1);
                        }
                    }
                    double* dst = sA + qq * sAq;
                    if (!TA) {
                        dst[pp * p.TM + ii] = v0;
                        if (ii + 1 < p.TM) dst[pp * p.TM + ii + 1] = v1;
                    } else {
                        if (pp < kc) dst[pp * p.TM + ii] = v0;
                        if (pp + 1 < kc) dst[(pp + 1) * p.TM + ii] = v1;
                    }
                }
            }
            // ---- pack op(B)(k0:k0+kc, j0:j0+TN), k-major, the same way (along j for B^T, along p
            // for B) ----
            {
                const int ext = TB ? p.TN : kc;
                const int hp = (ext + 1) >> 1;
                const int np2 = p.P * hp * (TB ? kc : p.TN);
                for (int e = t; e < np2; e += T) {
                    const int h = e % hp;
                    const int rest = e / hp;
                    int qq, pp, jj;
                    if (TB) {  // pair (jj, jj+1) in column k0 + pp of B^T's storage
                        jj = 2 * h;
                        pp = rest % kc;
                        qq = rest / kc;
                    } else {  // pair (pp, pp+1) of column j0 + jj
                        pp = 2 * h;
                        jj = rest % p.TN;
                        qq = rest / p.TN;
                    }
                    const long long qg = g * p.P + qq;
                    double v0 = 0.0, v1 = 0.0;
                    const int gj = j0 + jj;
                    const bool in0 = qg < p.batch && gj < p.n && (TB ? true : pp < kc);
                    const bool in1 = qg < p.batch && (TB ? (gj + 1 < p.n && jj + 1 < p.TN) : (gj < p.n && pp + 1 < kc));
                    if (in0) {
                        const double* Bq = p.B.ptr(qg);
                        const double* src = TB ? Bq + gj + (long long)(k0 + pp) * p.ldb
                                               : Bq + (k0 + pp) + (long long)gj * p.ldb;
                        if (in1 && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
                            const double2 w = ldg2(src);
                            v0 = w.x;
                            v1 = w.y;
                        } else {
                            v0 = ldg(src);
                            if (in1) v1 = ldg(src + 1);
                        }
                    }
                    double* dst = sB + qq * sBq;
                    if (TB) {
                        dst[pp * p.TN + jj] = v0;
                        if (jj + 1 < p.TN) dst[pp * p.TN + jj + 1] = v1;
                    } else {
                        if (pp < kc) dst[pp * p.TN + jj] = v0;
                        if (pp + 1 < kc) dst[(pp + 1) * p.TN + jj] = v1;
                    }
                }
            }
            __syncthreads();
            if (ql < p.P) {
                const double* a_s = sA + ql * sAq + ri;
                const double* b_s = sB + ql * sBq + rj;
#pragma unroll 2
                for (int pp = 0; pp < kc; pp++) {
                    double a[MR], bv[NR];
#pragma unroll
                    for (int s = 0; s < MR; s++) a[s] = a_s[pp * p.TM + GR * s];
#pragma unroll
                    for (int u = 0; u < NR; u++) bv[u] = b_s[pp * p.TN + GC * u];
#pragma unroll
                    for (int s = 0; s < MR; s++)
#pragma unroll
                        for (int u = 0; u < NR; u++)
                            acc[s][u] = NEG ? fma(-a[s], bv[u], acc[s][u]) : fma(a[s], bv[u], acc[s][u]);
                }
            }
            __syncthreads();
        }
    } else if (valid) {
        long long aoff[MR], boff[NR];
#pragma unroll
        for (int s = 0; s < MR; s++) aoff[s] = TA ? (long long)rc[s] * p.lda : rc[s];
#pragma unroll
        for (int u = 0; u < NR; u++) boff[u] = TB ? cc[u] : (long long)cc[u] * p.ldb;
        const long long astep = TA ? 1 : p.lda;
        const long long bstep = TB ? p.ldb : 1;
#pragma unroll 2
        for (int pp = 0; pp < p.k; pp++) {
            double a[MR], bv[NR];
#pragma unroll
            for (int s = 0; s < MR; s++) a[s] = ldg(A + aoff[s] + pp * astep);
#pragma unroll
            for (int u = 0; u < NR; u++) bv[u] = ldg(B + boff[u] + pp * bstep);
#pragma unroll
            for (int s = 0; s < MR; s++)
#pragma unroll
                for (int u = 0; u < NR; u++)
                    acc[s][u] = NEG ? fma(-a[s], bv[u], acc[s][u]) : fma(a[s], bv[u], acc[s][u]);
        }
    }

    if (!valid) return;
#pragma unroll
    for (int s = 0; s < MR; s++) {
#pragma unroll
        for (int u = 0; u < NR; u++) {
            const int i = rows[s], j = cols[u];
            if (i < p.m && j < p.n && in_tri(p.lower, i, j)) {
                double* cp = C + i + (long long)j * p.ldc;
                double v = acc[s][u];
                if (p.mode == ACC_GEN) v = (p.beta == 0.0) ? p.alpha * v : fma(p.alpha, v, p.beta * *cp);
                *cp = v;
            }
        }
    }
}

// C <= beta * C (alpha == 0 or k == 0); beta == 0 writes zeros without reading C.
__global__ void dscale_kernel(int m, int n, double beta, MatRef C, int ldc, long long batch) {
    const long long per = (long long)m * n;
    const long long total = per * batch;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long q = e / per;
        const long long r = e - q * per;
        const int j = (int)(r / m), i = (int)(r - (long long)j * m);
        double* cp = C.mptr(q) + i + (long long)j * ldc;
        *cp = (beta == 0.0) ? 0.0 : beta * *cp;
    }
}

template <int MR, int NR, bool PACKED, bool NEG>
static cudaError_t launch_t(const GemmParams& p, bool ta, bool tb, dim3 grid, dim3 block,
                            size_t smem, cudaStream_t s) {
#define BF_GEMM_CASE(A_, B_)                                                                 \
    if (ta == A_ && tb == B_) {                                                              \
        auto kfn = dgemm_tile_kernel<MR, NR, A_, B_, PACKED, NEG>;                            \
        if (smem + kStaticSmemSlack > 48 * 1024) {                                                              \
            cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                                 (int)smem);                                 \
            if (e != cudaSuccess) return e;                                                  \
        }                                                                                    \
        kfn<<<grid, block, smem, s>>>(p);                                                    \
        count_launch();                                                                      \
        return cudaGetLastError();                                                           \
    }
    BF_GEMM_CASE(false, false)
    BF_GEMM_CASE(false, true)
    BF_GEMM_CASE(true, false)
    BF_GEMM_CASE(true, true)
#undef BF_GEMM_CASE
    return cudaErrorInvalidValue;
}

size_t gemm_smem_bytes(const GemmConfig& c) {
    if (c.variant != VAR_PACKED) return 0;
    return sizeof(double) * ((size_t)c.P * ((size_t)c.KC * c.TM + 1) + (size_t)c.P * ((size_t)c.KC * c.TN + 1));
}

cudaError_t launch_dgemm(bool ta, bool tb, int m, int n, int k, double alpha, MatRef A, int lda,
                         MatRef B, int ldb, double beta, MatRef C, int ldc, long long batch,
                         const GemmConfig& cfg, int lower, const int* skip, cudaStream_t s) {
    if (m == 0 || n == 0 || batch == 0) return cudaSuccess;
    if (alpha == 0.0 || k == 0) {
        if (beta == 1.0) return cudaSuccess;
        long long total = (long long)m * n * batch;
        int blocks = (int)((total + 255) / 256);
        if (blocks > kSMs * 64) blocks = kSMs * 64;
        dscale_kernel<<<blocks, 256, 0, s>>>(m, n, beta, C, ldc, batch);
        count_launch();
        return cudaGetLastError();
    }
    if (cfg.variant == VAR_TINY && lower != TRI_NONE) {
        // the tiny kernel stores every entry of C: a triangle-masked product takes 4 x 4 direct tiles
        GemmConfig d = cfg;
        d.variant = VAR_DIRECT;
        d.TM = d.TN = 4;
        d.P = 64;
        return launch_dgemm(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, batch, d, lower, skip, s);
    }
    GemmParams p;
    p.m = m; p.n = n; p.k = k;
    p.alpha = alpha; p.beta = beta;
    p.mode = acc_mode(alpha == -1.0 ? 1.0 : alpha, beta);
    p.A = A; p.lda = lda; p.B = B; p.ldb = ldb; p.C = C; p.ldc = ldc;
    p.batch = batch;
    p.TM = cfg.TM; p.TN = cfg.TN; p.KC = cfg.KC; p.P = cfg.P;
    p.tilesM = (m + cfg.TM - 1) / cfg.TM;
    p.tilesN = (n + cfg.TN - 1) / cfg.TN;
    p.lower = lower;
    p.skip = skip;
    const bool neg = (alpha == -1.0);
    if (cfg.variant == VAR_TINY) return launch_dgemm_tiny(ta, tb, neg, p, s);
    const int tpp = (cfg.TM / 4) * (cfg.TN / 4);
    dim3 block(tpp * cfg.P);
    long long groups = (batch + cfg.P - 1) / cfg.P;
    dim3 grid((unsigned)(groups * p.tilesM * p.tilesN));
    size_t smem = gemm_smem_bytes(cfg);
    if (cfg.variant == VAR_PACKED)
        return neg ? launch_t<4, 4, true, true>(p, ta, tb, grid, block, smem, s)
                   : launch_t<4, 4, true, false>(p, ta, tb, grid, block, smem, s);
    return neg ? launch_t<4, 4, false, true>(p, ta, tb, grid, block, 0, s)
               : launch_t<4, 4, false, false>(p, ta, tb, grid, block, 0, s);
}

}  // namespace bf
