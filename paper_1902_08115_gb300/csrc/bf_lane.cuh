// bf_lane.cuh -- the lane Cholesky: one thread factors one whole problem.
//
// Left-looking by 4-column blocks, in the structure of the paper's
// kernel_dpotrf_nt_l (section 3.2.1): for the diagonal block a dgemm loop
// (D = A_JJ - L_J L_J^T), then a 4x4 Cholesky edge in registers; for every
// 4-row block below it a dgemm loop, then the triangular edge with the
// reciprocal pivots.  Shared by the uniform (bf_dpotrf.cu) and ragged
// (bf_ragged.cu) kernels.
//
// Operands are reached through an accessor.  ld4/st4 move a strip of four
// consecutive rows of one column (rows clamped to n - 1 on loads at the end
// of the matrix); the aligned global accessor does it with two 16-byte
// accesses, which halves the L1 requests of these uncoalesced per-lane
// streams (the lane kernels are bound by L1 request throughput, not DRAM).
#pragma once

#include "bf_common.cuh"

namespace bf {

struct GAcc {  // a problem in global memory
    double* a;
    int lda;
    __device__ __forceinline__ double ld(int i, int j) const { return a[i + (long long)j * lda]; }
    __device__ __forceinline__ void st(int i, int j, double v) const { a[i + (long long)j * lda] = v; }
    __device__ __forceinline__ void ld4(int i, int j, int n, double* o) const {
#pragma unroll
        for (int r = 0; r < 4; r++) o[r] = ld(imin(i + r, n - 1), j);
    }
    __device__ __forceinline__ void st4(int i, int j, int cnt, const double* v) const {
#pragma unroll
        for (int r = 0; r < 4; r++)
            if (r < cnt) st(i + r, j, v[r]);
    }
};

// Global memory, base 16-byte aligned and lda even: a strip starting at a row
// multiple of 4 is 16-byte aligned.
struct GAccV {
    double* a;
    int lda;
    __device__ __forceinline__ double ld(int i, int j) const { return a[i + (long long)j * lda]; }
    __device__ __forceinline__ void st(int i, int j, double v) const { a[i + (long long)j * lda] = v; }
    __device__ __forceinline__ void ld4(int i, int j, int n, double* o) const {
        if (i + 3 < n) {
            const double2* p = reinterpret_cast<const double2*>(a + i + (long long)j * lda);
            const double2 x = p[0], y = p[1];
            o[0] = x.x;
            o[1] = x.y;
            o[2] = y.x;
            o[3] = y.y;
        } else {
#pragma unroll
            for (int r = 0; r < 4; r++) o[r] = ld(imin(i + r, n - 1), j);
        }
    }
    __device__ __forceinline__ void st4(int i, int j, int cnt, const double* v) const {
        if (cnt == 4) {
            double2* p = reinterpret_cast<double2*>(a + i + (long long)j * lda);
            p[0] = make_double2(v[0], v[1]);
            p[1] = make_double2(v[2], v[3]);
        } else {
#pragma unroll
            for (int r = 0; r < 4; r++)
                if (r < cnt) st(i + r, j, v[r]);
        }
    }
};

struct SAcc {  // a problem in shared memory, interleaved with the CTA's other problems
    double* s;
    int n, T;
    __device__ __forceinline__ double ld(int i, int j) const { return s[(i + j * n) * T]; }
    __device__ __forceinline__ void st(int i, int j, double v) const { s[(i + j * n) * T] = v; }
    __device__ __forceinline__ void ld4(int i, int j, int nn, double* o) const {
#pragma unroll
        for (int r = 0; r < 4; r++) o[r] = ld(imin(i + r, nn - 1), j);
    }
    __device__ __forceinline__ void st4(int i, int j, int cnt, const double* v) const {
#pragma unroll
        for (int r = 0; r < 4; r++)
            if (r < cnt) st(i + r, j, v[r]);
    }
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
        for (int c = 0; c < 4; c++) {
            double col[4];
            M.ld4(J, jr[c], n, col);  // rows above c are read but not used (strict upper triangle)
#pragma unroll
            for (int r = c; r < 4; r++) d[r][c] = col[r];
        }
#pragma unroll 2
        for (int pp = 0; pp < J; pp++) {
            double l[4];
            M.ld4(J, pp, n, l);
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
        // lower part of the diagonal block only (the strict upper triangle is never written)
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c <= r; c++)
                if (r < jb) M.st(J + r, J + c, d[r][c]);
        // ---- 4-row blocks below: acc = A_IJ - L_I L_J^T, then acc L_JJ^{-T} ----
        for (int I = J + 4; I < n; I += 4) {
            const int ib = imin(4, n - I);
            double acc[4][4];
#pragma unroll
            for (int c = 0; c < 4; c++) {
                double col[4];
                M.ld4(I, jr[c], n, col);
#pragma unroll
                for (int r = 0; r < 4; r++) acc[r][c] = col[r];
            }
#pragma unroll 2
            for (int pp = 0; pp < J; pp++) {
                double a[4], b[4];
                M.ld4(I, pp, n, a);
                M.ld4(J, pp, n, b);
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
            for (int c = 0; c < 4; c++) {
                if (c < jb) {
                    double col[4];
#pragma unroll
                    for (int r = 0; r < 4; r++) col[r] = acc[r][c];
                    M.st4(I, J + c, ib, col);
                }
            }
        }
    }
    return 0;
}

// 16-byte alignment of every 4-row strip: base aligned and lda even
__device__ __forceinline__ bool strips_aligned(const double* a, int lda) {
    return ((reinterpret_cast<unsigned long long>(a) & 15ull) == 0) && ((lda & 1) == 0);
}

}  // namespace bf
