// bf_dtrsm.cu -- batched FP64 triangular solve (section 3.1 "dtrsm").
//
// The paper implements only the right-side kernels, because they solve many
// small independent row systems with the triangle broadcast (vector
// friendly), and obtains the left side by transposition:
// op(A)^{-1} B = (B^T op(A)^{-T})^T (section 3.1 "dtrsm").  The same holds on
// the GPU: every row of the right-hand side is an independent system, so one
// thread solves MR rows and all threads of a warp run the same instruction
// stream.  A left solve is the right solve of B^T against op(A)^T, i.e. the
// same kernel reading B transposed ("bt") and A with the opposite transpose.
//
// Kernel structure per 4-column block J (the paper's dtrsm kernel: a dgemm
// loop followed by a register-resident triangular edge):
//   acc = alpha R(rows, J)  -  X(rows, solved) T(solved, J)     (dgemm loop)
//   acc = acc T(J, J)^{-1}                                       (edge, in registers)
//   R(rows, J) = acc                                             (store)
// T upper is solved forward (j = 0..n-1), T lower backward (j = n-1..0).
#include "bf_internal.h"

namespace bf {

// MINB: CTAs of 256 threads the kernel is compiled to keep resident per SM (2 caps the
// registers at 128).
// UNIT: unit diagonal (no reciprocal pivots; the kernel carries none of their code).
template <int MR, bool PACKED, bool UP, int MINB, bool UNIT>
__global__ void __launch_bounds__(256, MINB)
dtrsm_rows_kernel(TrsmParams p) {
    extern __shared__ double smem[];
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long q = gt / p.tpp;
    const int rr = (int)(gt - q * p.tpp);
    const int n = p.n;
    // PACKED: the CTA's problems' triangles and reciprocal diagonals in shared memory
    const long long q0 = (blockIdx.x * (long long)blockDim.x) / p.tpp;
    const int ldt = n + 1;
    double* sT = smem;
    double* sR = smem + (size_t)p.P * n * ldt;
    if (PACKED) {
        const int per = n * n;
        for (int e = threadIdx.x; e < p.P * per; e += blockDim.x) {
            const int qq = e / per;
            const int rem = e - qq * per;
            const int j = rem / n, i = rem - j * n;
            const long long qg = q0 + qq;
            double v = 0.0;
            const bool inT = UP ? (i <= j) : (i >= j);
            if (qg < p.batch && inT && !(UNIT && i == j)) {
                const double* Aq = p.A.ptr(qg);
                v = p.et ? ldg(Aq + j + (long long)i * p.lda) : ldg(Aq + i + (long long)j * p.lda);
            }
            sT[qq * n * ldt + i + j * ldt] = v;  // sT(i, j) = T(i, j)
        }
        __syncthreads();
        if (!UNIT) {
            for (int e = threadIdx.x; e < p.P * n; e += blockDim.x) {
                const int qq = e / n, j = e - (e / n) * n;
                sR[qq * n + j] = 1.0 / sT[qq * n * ldt + j + j * ldt];
            }
            __syncthreads();
        }
    }
    if (q >= p.batch) return;
    if (p.skip && p.skip[q] != 0) return;

    const double* A = p.A.ptr(q);
    double* B = p.B.mptr(q);
    const double* Ts = PACKED ? (sT + (q - q0) * n * ldt) : nullptr;
    const double* Rs = PACKED ? (sR + (q - q0) * n) : nullptr;

    int rows[MR];
    int roff[MR];  // element offsets within the problem (a small matrix: 32 bits suffice)
#pragma unroll
    for (int s = 0; s < MR; s++) {
        rows[s] = rr + p.tpp * s;
        const int rc = imin(rows[s], p.m - 1);
        roff[s] = p.bt ? rc * p.ldb : rc;
    }
    const long long cstep = p.bt ? 1 : p.ldb;  // R(r, j + 1) - R(r, j)

    auto Tel = [&](int i, int j) -> double {
        if (PACKED) return Ts[i + j * ldt];
        return p.et ? ldg(A + j + (long long)i * p.lda) : ldg(A + i + (long long)j * p.lda);
    };

    // reciprocal pivots shared over a problem's lanes when they sit in one warp (tpp a power of
    // two up to 32: problems then start on multiples of tpp within a warp)
    const bool share = !PACKED && p.tpp > 1 && p.tpp <= 32 && (p.tpp & (p.tpp - 1)) == 0;
    const int nblk = (n + 3) / 4;
    for (int bi = 0; bi < nblk; bi++) {
        const int blk = UP ? bi : (nblk - 1 - bi);
        const int J = blk * 4;
        const int jb = imin(4, n - J);
        double acc[MR][4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int jc = imin(J + c, n - 1);
#pragma unroll
            for (int s = 0; s < MR; s++) acc[s][c] = B[roff[s] + jc * cstep];
        }
        if (p.alpha != 1.0) {
#pragma unroll
            for (int s = 0; s < MR; s++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[s][c] *= p.alpha;
        }
        // dgemm loop over the already solved columns
        const int pb = UP ? 0 : J + jb;
        const int pe = UP ? J : n;
#pragma unroll 2
        for (int pp = pb; pp < pe; pp++) {
            double x[MR], tv[4];
#pragma unroll
            for (int s = 0; s < MR; s++) x[s] = B[roff[s] + pp * cstep];
#pragma unroll
            for (int c = 0; c < 4; c++) tv[c] = Tel(pp, imin(J + c, n - 1));
#pragma unroll
            for (int s = 0; s < MR; s++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[s][c] = fma(-x[s], tv[c], acc[s][c]);
        }
        // triangular edge on the jb x jb diagonal block, in registers
        double tb[4][4], rinv[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
#pragma unroll
            for (int c2 = 0; c2 < 4; c2++) {
                const bool need = UP ? (c2 < c) : (c2 > c);
                tb[c2][c] = (need && c < jb && c2 < jb) ? Tel(J + c2, J + c) : 0.0;
            }
        }
        if (!UNIT) {
            if (PACKED) {
#pragma unroll
                for (int c = 0; c < 4; c++) rinv[c] = (c < jb) ? Rs[J + c] : 1.0;
            } else if (share) {
                // the problem's tpp lanes (adjacent, one warp) split the four reciprocals and
                // exchange them: lane rr takes columns rr, rr + tpp, ...
                double own[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int c = rr + k * p.tpp;
                    own[k] = 1.0;
                    if (k * p.tpp < 4 && c < jb) own[k] = 1.0 / Tel(J + c, J + c);
                }
                const unsigned mask = __activemask();
                const int base = (threadIdx.x & 31) - rr;
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    double v = own[0];
#pragma unroll
                    for (int k = 1; k < 4; k++)
                        if (c / p.tpp == k) v = own[k];
                    rinv[c] = __shfl_sync(mask, v, base + c % p.tpp);
                }
            } else {
#pragma unroll
                for (int c = 0; c < 4; c++) rinv[c] = (c < jb) ? 1.0 / Tel(J + c, J + c) : 1.0;
            }
        }
        if (UP) {
#pragma unroll
            for (int c = 0; c < 4; c++) {
#pragma unroll
                for (int c2 = 0; c2 < c; c2++)
#pragma unroll
                    for (int s = 0; s < MR; s++) acc[s][c] = fma(-acc[s][c2], tb[c2][c], acc[s][c]);
                if (!UNIT)
#pragma unroll
                    for (int s = 0; s < MR; s++) acc[s][c] *= rinv[c];
            }
        } else {
#pragma unroll
            for (int c = 3; c >= 0; c--) {
#pragma unroll
                for (int c2 = c + 1; c2 < 4; c2++)
#pragma unroll
                    for (int s = 0; s < MR; s++) acc[s][c] = fma(-acc[s][c2], tb[c2][c], acc[s][c]);
                if (!UNIT)
#pragma unroll
                    for (int s = 0; s < MR; s++) acc[s][c] *= rinv[c];
            }
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
            if (c < jb) {
#pragma unroll
                for (int s = 0; s < MR; s++)
                    if (rows[s] < p.m) B[roff[s] + (J + c) * cstep] = acc[s][c];
            }
        }
    }
}

template <int MR, bool PACKED, bool UP>
static cudaError_t launch_rows3(const TrsmParams& p, long long threads, int block, size_t smem, int minb,
                               cudaStream_t s) {
    // the residency is a tuned choice: with few, large problems one more CTA per SM can
    // decide whether the launch fits one wave (or how full its last wave is)
    auto kfn = p.unit ? ((!PACKED && minb == 2) ? dtrsm_rows_kernel<MR, PACKED, UP, 2, true>
                                                : dtrsm_rows_kernel<MR, PACKED, UP, 1, true>)
                      : ((!PACKED && minb == 2) ? dtrsm_rows_kernel<MR, PACKED, UP, 2, false>
                                                : dtrsm_rows_kernel<MR, PACKED, UP, 1, false>);
    if (smem + kStaticSmemSlack > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    long long blocks = (threads + block - 1) / block;
    kfn<<<(unsigned)blocks, block, smem, s>>>(p);
    count_launch();
    return cudaGetLastError();
}

template <int MR, bool PACKED>
static cudaError_t launch_rows(const TrsmParams& p, long long threads, int block, size_t smem, int minb,
                               cudaStream_t s) {
    return p.upper ? launch_rows3<MR, PACKED, true>(p, threads, block, smem, minb, s)
                   : launch_rows3<MR, PACKED, false>(p, threads, block, smem, minb, s);
}

static cudaError_t launch_dtrsm_blocked(int side, int uplo, int trans, int unit, int m, int n, double alpha,
                                        MatRef A, int lda, MatRef B, int ldb, long long batch, int NB,
                                        const int* skip, cudaStream_t s);

cudaError_t launch_dtrsm(int side, int uplo, int trans, int unit, int m, int n, double alpha,
                         MatRef A, int lda, MatRef B, int ldb, long long batch,
                         const TrsmConfig& cfg, const int* skip, cudaStream_t s) {
    if (m == 0 || n == 0 || batch == 0) return cudaSuccess;
    if (cfg.variant == VAR_BLOCKED && alpha != 0.0)
        return launch_dtrsm_blocked(side, uplo, trans, unit, m, n, alpha, A, lda, B, ldb, batch, 32, skip, s);
    if (cfg.variant == VAR_BLOCKED) {  // alpha == 0: B = 0, A not read (the row kernel's path)
        TrsmConfig d = cfg;
        d.variant = VAR_DIRECT;
        d.P = 1;
        return launch_dtrsm(side, uplo, trans, unit, m, n, alpha, A, lda, B, ldb, batch, d, skip, s);
    }
    if (cfg.variant == VAR_TINY) return launch_dtrsm_tiny(side, uplo, trans, unit, m, n, alpha, A, lda, B, ldb, batch,
                                                          skip, s);
    TrsmParams p;
    const bool right = (side == 1);
    // rows of R: right -> rows of B (m x n, T is n x n); left -> columns of B (R = B^T, T is m x m)
    p.m = right ? m : n;
    p.n = right ? n : m;
    p.alpha = alpha;
    p.A = A; p.lda = lda; p.B = B; p.ldb = ldb;
    p.batch = batch;
    p.bt = right ? 0 : 1;
    p.et = right ? trans : !trans;
    p.upper = (uplo == 1) ^ p.et;
    p.unit = unit;
    p.skip = skip;
    const int MR = cfg.MR;
    p.tpp = (p.m + MR - 1) / MR;
    long long threads = batch * p.tpp;
    if (cfg.variant == VAR_PACKED) {
        // one CTA holds P whole problems (block = P * tpp threads)
        p.P = cfg.P;
        int block = p.P * p.tpp;
        size_t smem = sizeof(double) * ((size_t)p.P * p.n * (p.n + 1) + (size_t)p.P * p.n);
        threads = ((batch + p.P - 1) / p.P) * (long long)block;
        return MR == 8 ? launch_rows<8, true>(p, threads, block, smem, 1, s)
                       : launch_rows<4, true>(p, threads, block, smem, 1, s);
    }
    p.P = 1;
    // fewer than 256 threads per CTA when the rows are few (a small batch, or a block of the
    // blocked form), so that every SM still gets work
    const int block = spread_block(threads, 256);
    return MR == 8 ? launch_rows<8, false>(p, threads, block, 0, cfg.minb, s)
                   : launch_rows<4, false>(p, threads, block, 0, cfg.minb, s);
}

// Blocked triangular solve for batches too small to fill the GPU with one thread per row:
// the blocks of NB rows/columns of op(A) in solve order, each a row-parallel solve against its
// diagonal block, followed by a dgemm that removes the block's contribution from the blocks
// still to solve (the paper's dtrsm kernel, a dgemm loop plus a triangular edge, with the
// dgemm loop hoisted out as a batched dgemm with 2-D parallelism).  alpha scales the first
// block's solve and, through the first update's beta, every block after it.
static cudaError_t launch_dtrsm_blocked(int side, int uplo, int trans, int unit, int m, int n, double alpha,
                                        MatRef A, int lda, MatRef B, int ldb, long long batch, int NB,
                                        const int* skip, cudaStream_t s) {
    const bool right = side == 1;
    const int order = right ? n : m;
    const bool lowerT = (uplo == 0) != (trans != 0);  // op(A) lower
    const bool fwd = right ? !lowerT : lowerT;        // blocks in ascending order
    const int nblk = (order + NB - 1) / NB;
    for (int t = 0; t < nblk; t++) {
        const int bi = fwd ? t : nblk - 1 - t;
        const int J = bi * NB, jb = (order - J < NB) ? order - J : NB;
        const double a = t == 0 ? alpha : 1.0;
        const int mm = right ? m : jb, nn = right ? jb : n;
        const MatRef Bj = right ? mat_sub(B, 0, J, ldb) : mat_sub(B, J, 0, ldb);
        TrsmConfig c = choose_trsm(side, uplo, trans, unit, mm, nn, 1LL << 40);  // the row kernel's table entry
        cudaError_t e = launch_dtrsm(side, uplo, trans, unit, mm, nn, a, mat_sub(A, J, J, lda), lda, Bj, ldb, batch,
                                     c, skip, s);
        if (e != cudaSuccess) return e;
        const int rlo = fwd ? J + jb : 0, rn = fwd ? order - J - jb : J;  // the blocks still to solve
        if (rn <= 0) continue;
        const double beta = t == 0 ? alpha : 1.0;
        if (right) {
            // B(:, rest) = beta B(:, rest) - X_J op(A)(J, rest); op(A)(J, rest) = A(J, rest) or A(rest, J)^T
            const MatRef opA = trans ? mat_sub(A, rlo, J, lda) : mat_sub(A, J, rlo, lda);
            GemmConfig g = choose_gemm(false, trans != 0, m, rn, jb, ldb, batch);
            e = launch_dgemm(false, trans != 0, m, rn, jb, -1.0, Bj, ldb, opA, lda, beta, mat_sub(B, 0, rlo, ldb), ldb,
                             batch, g, 0, skip, s);
        } else {
            // B(rest, :) = beta B(rest, :) - op(A)(rest, J) X_J; op(A)(rest, J) = A(rest, J) or A(J, rest)^T
            const MatRef opA = trans ? mat_sub(A, J, rlo, lda) : mat_sub(A, rlo, J, lda);
            GemmConfig g = choose_gemm(trans != 0, false, rn, n, jb, lda, batch);
            e = launch_dgemm(trans != 0, false, rn, n, jb, -1.0, opA, lda, Bj, ldb, beta, mat_sub(B, rlo, 0, ldb), ldb,
                             batch, g, 0, skip, s);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace bf
