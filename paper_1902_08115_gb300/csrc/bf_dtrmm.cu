// bf_dtrmm.cu -- batched FP64 triangular multiply (section 3.1 "dtrmm": the same
// considerations as dtrsm), B <= alpha op(A) B (left) or alpha B op(A) (right).
//
// As for dtrsm, only the right side has a kernel: every row of B is transformed
// independently, b <= alpha b T with T = op(A) triangular, so one thread owns MR rows and
// the warp runs one instruction stream.  The left side is the right side of B^T against
// op(A)^T (B read transposed, A with the opposite transpose).  The multiply is done in
// place, 4 columns at a time, in the order that leaves every column still needed
// unwritten: for T lower, new column j uses old columns j..n-1, so blocks go left to right;
// for T upper, new column j uses old columns 0..j, so blocks go right to left.  Per block J:
//   acc  = B(rows, outside J) T(outside J, J)        (dgemm loop over the untouched columns)
//   acc += B(rows, J) T(J, J)                        (triangular edge; unit diagonal = 1)
//   B(rows, J) = alpha acc
#include "bf_internal.h"

namespace bf {

template <int MR, bool SRC>
__global__ void __launch_bounds__(256) dtrmm_rows_kernel(TrsmParams p) {
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long q = gt / p.tpp;
    const int rr = (int)(gt - q * p.tpp);
    if (q >= p.batch) return;
    const int n = p.n;
    const double* A = p.A.ptr(q);
    double* B = p.B.mptr(q);
    // SRC (out of place): the old values come from Bsrc, so the block order no longer matters
    const double* Bs = SRC ? p.Bsrc.ptr(q) : B;
    const int ldbs = SRC ? p.ldbs : p.ldb;
    int rows[MR];
    long long roff[MR], roffs[MR];
#pragma unroll
    for (int s = 0; s < MR; s++) {
        rows[s] = rr + p.tpp * s;
        const int rc = imin(rows[s], p.m - 1);
        roff[s] = p.bt ? (long long)rc * p.ldb : rc;
        roffs[s] = SRC ? (p.bt ? (long long)rc * ldbs : rc) : roff[s];
    }
    const long long cstep = p.bt ? 1 : p.ldb;  // R(r, j + 1) - R(r, j)
    const long long csteps = SRC ? (p.bt ? 1 : ldbs) : cstep;
    auto Tel = [&](int i, int j) -> double {
        return p.et ? ldg(A + j + (long long)i * p.lda) : ldg(A + i + (long long)j * p.lda);
    };
    const int nblk = (n + 3) / 4;
    for (int bi = 0; bi < nblk; bi++) {
        const int blk = p.upper ? (nblk - 1 - bi) : bi;
        const int J = blk * 4;
        const int jb = imin(4, n - J);
        double acc[MR][4];
#pragma unroll
        for (int s = 0; s < MR; s++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[s][c] = 0.0;
        // columns outside the block that still hold their old values
        const int pb = p.upper ? 0 : J + jb;
        const int pe = p.upper ? J : n;
#pragma unroll 2
        for (int pp = pb; pp < pe; pp++) {
            double x[MR], tv[4];
#pragma unroll
            for (int s = 0; s < MR; s++) x[s] = Bs[roffs[s] + pp * csteps];
#pragma unroll
            for (int c = 0; c < 4; c++) tv[c] = Tel(pp, imin(J + c, n - 1));
#pragma unroll
            for (int s = 0; s < MR; s++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[s][c] = fma(x[s], tv[c], acc[s][c]);
        }
        // the block's own columns through the jb x jb triangle
        double xb[MR][4], tb[4][4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int jc = imin(J + c, n - 1);
#pragma unroll
            for (int s = 0; s < MR; s++) xb[s][c] = Bs[roffs[s] + jc * csteps];
        }
#pragma unroll
        for (int c = 0; c < 4; c++)
#pragma unroll
            for (int c2 = 0; c2 < 4; c2++) {
                const bool in = p.upper ? (c2 <= c) : (c2 >= c);
                double v = 0.0;
                if (in && c < jb && c2 < jb) v = (c2 == c && p.unit) ? 1.0 : Tel(J + c2, J + c);
                tb[c2][c] = v;
            }
#pragma unroll
        for (int c = 0; c < 4; c++)
#pragma unroll
            for (int c2 = 0; c2 < 4; c2++)
#pragma unroll
                for (int s = 0; s < MR; s++) acc[s][c] = fma(xb[s][c2], tb[c2][c], acc[s][c]);
#pragma unroll
        for (int c = 0; c < 4; c++) {
            if (c < jb) {
#pragma unroll
                for (int s = 0; s < MR; s++)
                    if (rows[s] < p.m) B[roff[s] + (J + c) * cstep] = p.alpha * acc[s][c];
            }
        }
    }
}

cudaError_t launch_dtrmm(int side, int uplo, int trans, int unit, int m, int n, double alpha, MatRef A, int lda,
                         MatRef B, int ldb, long long batch, int MR, cudaStream_t s, const MatRef* Bsrc, int ldbs) {
    if (m == 0 || n == 0 || batch == 0) return cudaSuccess;
    TrsmParams p;
    if (Bsrc) {
        p.Bsrc = *Bsrc;
        p.ldbs = ldbs;
        p.has_src = 1;
    }
    const bool right = (side == 1);
    // rows of R: right -> rows of B (T = op(A) is n x n); left -> columns of B (R = B^T, T = op(A)^T)
    p.m = right ? m : n;
    p.n = right ? n : m;
    p.alpha = alpha;
    p.A = A; p.lda = lda; p.B = B; p.ldb = ldb;
    p.batch = batch;
    p.bt = right ? 0 : 1;
    p.et = right ? trans : !trans;
    p.upper = (uplo == 1) ^ p.et;
    p.unit = unit;
    p.skip = nullptr;
    p.P = 1;
    MR = (MR == 8) ? 8 : 4;
    p.tpp = (p.m + MR - 1) / MR;
    const long long threads = batch * p.tpp;
    const int T = 256;
    const unsigned blocks = (unsigned)((threads + T - 1) / T);
    if (p.has_src) {
        if (MR == 8) dtrmm_rows_kernel<8, true><<<blocks, T, 0, s>>>(p);
        else dtrmm_rows_kernel<4, true><<<blocks, T, 0, s>>>(p);
    } else {
        if (MR == 8) dtrmm_rows_kernel<8, false><<<blocks, T, 0, s>>>(p);
        else dtrmm_rows_kernel<4, false><<<blocks, T, 0, s>>>(p);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace bf
