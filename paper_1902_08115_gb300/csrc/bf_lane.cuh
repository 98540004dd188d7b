// bf_lane.cuh -- the lane Cholesky: one thread factors one whole problem.
//
// Left-looking by 4-column blocks, in the structure of the paper's
// kernel_dpotrf_nt_l (section 3.2.1): for the diagonal block a dgemm loop
// (D = A_JJ - L_J L_J^T), then a 4x4 Cholesky edge in registers; for every
// 4-row block below it a dgemm loop, then the triangular edge with the
// reciprocal pivots.  Shared by the uniform (bf_dpotrf.cu) and ragged
// (bf_ragged.cu) kernels.
#pragma once

#include "bf_common.cuh"

namespace bf {

struct GAcc {  // a problem in global memory
    double* a;
    int lda;
    __device__ __forceinline__ double ld(int i, int j) const { return a[i + (long long)j * lda]; }
    __device__ __forceinline__ void st(int i, int j, double v) const { a[i + (long long)j * lda] = v; }
};

struct SAcc {  // a problem in shared memory, interleaved with the CTA's other problems
    double* s;
    int n, T;
    __device__ __forceinline__ double ld(int i, int j) const { return s[(i + j * n) * T]; }
    __device__ __forceinline__ void st(int i, int j, double v) const { s[(i + j * n) * T] = v; }
};

// Factor one problem in place through the accessor.  Returns info (0 or 1-based column).
template <class Acc>
__device__ __forceinline__ int potrf_lane(const Acc& M, int n) {
    for (int J = 0; J < n; J += 4) {
        const int jb = imin(4, n - J);
        int jr[4];
#pragma unroll
        for (int r = 0; r < 4; r++) jr[r] = imin(J + r, n - 1);
        // ---- diagonal block: D = A_JJ - sum_p L(J:J+4, p) L(J:J+4, p)^T (lower part) ----
        double d[4][4];
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c <= r; c++) d[r][c] = M.ld(jr[r], jr[c]);
        for (int pp = 0; pp < J; pp++) {
            double l[4];
#pragma unroll
            for (int r = 0; r < 4; r++) l[r] = M.ld(jr[r], pp);
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c <= r; c++) d[r][c] = fma(-l[r], l[c], d[r][c]);
        }
        // pad the block beyond n with the identity
#pragma unroll
        for (int r = 0; r < 4; r++) {
            if (r >= jb) {
#pragma unroll
                for (int c = 0; c < r; c++) d[r][c] = 0.0;
                d[r][r] = 1.0;
            }
        }
        // ---- 4x4 Cholesky edge in registers ----
        double rinv[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const double piv = d[c][c];
            if (!(piv > 0.0)) return J + c + 1;
            const double rs = rsqrt(piv);
            rinv[c] = rs;
            d[c][c] = piv * rs;
#pragma unroll
            for (int r = c + 1; r < 4; r++) d[r][c] *= rs;
#pragma unroll
            for (int r = c + 1; r < 4; r++)
#pragma unroll
                for (int c2 = c + 1; c2 <= r; c2++) d[r][c2] = fma(-d[r][c], d[c2][c], d[r][c2]);
        }
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c <= r; c++)
                if (r < jb) M.st(J + r, J + c, d[r][c]);
        // ---- 4-row blocks below: acc = A_IJ - L_I L_J^T, then acc L_JJ^{-T} ----
        for (int I = J + 4; I < n; I += 4) {
            const int ib = imin(4, n - I);
            int ir[4];
#pragma unroll
            for (int r = 0; r < 4; r++) ir[r] = imin(I + r, n - 1);
            double acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[r][c] = M.ld(ir[r], jr[c]);
            for (int pp = 0; pp < J; pp++) {
                double a[4], b[4];
#pragma unroll
                for (int r = 0; r < 4; r++) a[r] = M.ld(ir[r], pp);
#pragma unroll
                for (int c = 0; c < 4; c++) b[c] = M.ld(jr[c], pp);
#pragma unroll
                for (int r = 0; r < 4; r++)
#pragma unroll
                    for (int c = 0; c < 4; c++) acc[r][c] = fma(-a[r], b[c], acc[r][c]);
            }
#pragma unroll
            for (int c = 0; c < 4; c++) {
#pragma unroll
                for (int c2 = 0; c2 < c; c2++)
#pragma unroll
                    for (int r = 0; r < 4; r++) acc[r][c] = fma(-acc[r][c2], d[c][c2], acc[r][c]);
#pragma unroll
                for (int r = 0; r < 4; r++) acc[r][c] *= rinv[c];
            }
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++)
                    if (r < ib && c < jb) M.st(I + r, J + c, acc[r][c]);
        }
    }
    return 0;
}

}  // namespace bf
