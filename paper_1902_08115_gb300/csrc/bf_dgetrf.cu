// bf_dgetrf.cu -- batched FP64 LU factorisation with partial (row) pivoting, P A = L U
// (section 3.1 "dgetrf"), and the solve dgetrs.
//
// The paper computes dgetrf by column blocks, packing each column block into row-major
// panels so that the dgemm_nt kernel and right-hand triangular solves apply (section 3.1
// "dgetrf").  Here one thread factors one whole square problem (the lane form of the
// Cholesky kernels: the 32 lanes of a warp run 32 problems' identical instruction streams,
// and a masked FP64 lane costs a full one), left-looking by 4-column blocks J:
//   (1) U(0:J, J:J+4) = L(0:J, 0:J)^{-1} A(0:J, J:J+4)   (unit lower forward substitution,
//       4x4 register tiles: dgemm loop + triangular edge)
//   (2) A(J:n, J:J+4) -= L(J:n, 0:J) U(0:J, J:J+4)      (dgemm loop, 4x4 register tiles)
//   (3) the n-J x 4 panel factored column by column: pivot = the first row of largest |a|
//       (a NaN never counts as larger), the two rows swapped across all n columns, the
//       column below scaled by the pivot's reciprocal, the panel's later columns updated.
// Rows are swapped eagerly, so every column still to be processed already holds P A.
// info = the first column whose pivot is exactly zero (the factorisation still completes,
// as LAPACK's); ipiv is 1-based.
#include "bf_internal.h"
#include "bf_lane.cuh"

namespace bf {

struct GetrfParams {
    int n;
    MatRef A;
    int lda;
    int* ipiv;
    long long sipiv;
    long long batch;
    int* info;
};

template <class Acc>
__device__ __forceinline__ int getrf_lane(const Acc& M, int n, int* piv) {
    int info = 0;
    for (int J = 0; J < n; J += 4) {
        const int jb = imin(4, n - J);
        int jc[4];
#pragma unroll
        for (int c = 0; c < 4; c++) jc[c] = imin(J + c, n - 1);
        // (1) rows 0..J of the block column: unit lower forward substitution
        for (int I = 0; I < J; I += 4) {
            double acc[4][4];
#pragma unroll
            for (int c = 0; c < 4; c++) {
                double col[4];
                M.template strip<4>(I, jc[c], n, col);
#pragma unroll
                for (int r = 0; r < 4; r++) acc[r][c] = col[r];
            }
#pragma unroll 2
            for (int p = 0; p < I; p++) {
                double l[4], u[4];
                M.template strip<4>(I, p, n, l);
#pragma unroll
                for (int c = 0; c < 4; c++) u[c] = M.ld(p, jc[c]);
#pragma unroll
                for (int r = 0; r < 4; r++)
#pragma unroll
                    for (int c = 0; c < 4; c++) acc[r][c] = fma(-l[r], u[c], acc[r][c]);
            }
            double lt[4][4];  // the block's unit lower triangle (I + 3 < J <= n)
#pragma unroll
            for (int r = 1; r < 4; r++)
#pragma unroll
                for (int r2 = 0; r2 < r; r2++) lt[r][r2] = M.ld(I + r, I + r2);
#pragma unroll
            for (int r = 1; r < 4; r++)
#pragma unroll
                for (int r2 = 0; r2 < r; r2++)
#pragma unroll
                    for (int c = 0; c < 4; c++) acc[r][c] = fma(-lt[r][r2], acc[r2][c], acc[r][c]);
#pragma unroll
            for (int c = 0; c < 4; c++) {
                if (c < jb) {
                    double col[4];
#pragma unroll
                    for (int r = 0; r < 4; r++) col[r] = acc[r][c];
                    M.template put<4>(I, J + c, 4, col);
                }
            }
        }
        // (2) rows J..n-1 of the block column: subtract L(J:n, 0:J) U(0:J, J:J+4)
        if (J > 0) {
            for (int I = J; I < n; I += 4) {
                double acc[4][4];
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    double col[4];
                    M.template strip<4>(I, jc[c], n, col);
#pragma unroll
                    for (int r = 0; r < 4; r++) acc[r][c] = col[r];
                }
#pragma unroll 2
                for (int p = 0; p < J; p++) {
                    double l[4], u[4];
                    M.template strip<4>(I, p, n, l);
#pragma unroll
                    for (int c = 0; c < 4; c++) u[c] = M.ld(p, jc[c]);
#pragma unroll
                    for (int r = 0; r < 4; r++)
#pragma unroll
                        for (int c = 0; c < 4; c++) acc[r][c] = fma(-l[r], u[c], acc[r][c]);
                }
                const int ib = imin(4, n - I);
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    if (c < jb) {
                        double col[4];
#pragma unroll
                        for (int r = 0; r < 4; r++) col[r] = acc[r][c];
                        M.template put<4>(I, J + c, ib, col);
                    }
                }
            }
        }
        // (3) the panel, column by column, with partial pivoting
        for (int c = 0; c < jb; c++) {
            const int col = J + c;
            int p = col;
            double best = fabs(M.ld(col, col));
            for (int i = col + 1; i < n; i++) {
                const double v = fabs(M.ld(i, col));
                if (v > best) {
                    best = v;
                    p = i;
                }
            }
            piv[col] = p + 1;
            const double pv = M.ld(p, col);
            if (pv != 0.0) {
                if (p != col) {
                    for (int k = 0; k < n; k++) {
                        const double t = M.ld(col, k);
                        M.st(col, k, M.ld(p, k));
                        M.st(p, k, t);
                    }
                }
                const double rcp = 1.0 / pv;
                for (int i = col + 1; i < n; i++) M.st(i, col, M.ld(i, col) * rcp);
            } else if (info == 0) {
                info = col + 1;
            }
            for (int c2 = c + 1; c2 < jb; c2++) {
                const double u = M.ld(col, J + c2);
                for (int i = col + 1; i < n; i++) M.st(i, J + c2, fma(-M.ld(i, col), u, M.ld(i, J + c2)));
            }
        }
    }
    return info;
}

__global__ void __launch_bounds__(256) dgetrf_lane_kernel(GetrfParams p) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= p.batch) return;
    double* a = p.A.mptr(q);
    int* piv = p.ipiv + q * p.sipiv;
    const int info = strips_aligned(a, p.lda) ? getrf_lane(GAccV{a, p.lda}, p.n, piv)
                                              : getrf_lane(GAccP{a, p.lda}, p.n, piv);
    if (p.info) p.info[q] = info;
}

cudaError_t launch_dgetrf(int n, MatRef A, int lda, int* ipiv, long long sipiv, int* info, long long batch,
                          cudaStream_t s) {
    if (batch == 0) return cudaSuccess;
    if (n == 0) return info ? cudaMemsetAsync(info, 0, sizeof(int) * (size_t)batch, s) : cudaSuccess;
    GetrfParams p;
    p.n = n; p.A = A; p.lda = lda; p.ipiv = ipiv; p.sipiv = sipiv; p.batch = batch; p.info = info;
    const int T = 64;
    dgetrf_lane_kernel<<<(unsigned)((batch + T - 1) / T), T, 0, s>>>(p);
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ dgetrs
// the row interchanges of ipiv applied to B (n x nrhs): forward (j ascending) for 'N',
// backward (j descending) after the solves for 'T'; one thread per (problem, column)
__global__ void laswp_kernel(int n, int nrhs, MatRef B, int ldb, const int* ipiv, long long sipiv, int backward,
                             long long batch) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long q = g / nrhs;
    if (q >= batch) return;
    const int c = (int)(g - q * nrhs);
    double* b = B.mptr(q) + (long long)c * ldb;
    const int* piv = ipiv + q * sipiv;
    for (int t = 0; t < n; t++) {
        const int j = backward ? n - 1 - t : t;
        const int pj = piv[j] - 1;
        if (pj != j) {
            const double x = b[j];
            b[j] = b[pj];
            b[pj] = x;
        }
    }
}

cudaError_t launch_dgetrs(int trans, int n, int nrhs, MatRef A, int lda, const int* ipiv, long long sipiv, MatRef B,
                          int ldb, long long batch, cudaStream_t s) {
    if (n == 0 || nrhs == 0 || batch == 0) return cudaSuccess;
    const long long threads = batch * nrhs;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    cudaError_t e;
    if (!trans) {
        laswp_kernel<<<blocks, 256, 0, s>>>(n, nrhs, B, ldb, ipiv, sipiv, 0, batch);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // L Y = P B (unit lower), then U X = Y
        TrsmConfig c1 = choose_trsm(0, 0, 0, 1, n, nrhs, batch);
        if ((e = launch_dtrsm(0, 0, 0, 1, n, nrhs, 1.0, A, lda, B, ldb, batch, c1, nullptr, s)) != cudaSuccess)
            return e;
        TrsmConfig c2 = choose_trsm(0, 1, 0, 0, n, nrhs, batch);
        return launch_dtrsm(0, 1, 0, 0, n, nrhs, 1.0, A, lda, B, ldb, batch, c2, nullptr, s);
    }
    // U^T Y = B, L^T Z = Y (unit), then the interchanges in reverse order
    TrsmConfig c1 = choose_trsm(0, 1, 1, 0, n, nrhs, batch);
    if ((e = launch_dtrsm(0, 1, 1, 0, n, nrhs, 1.0, A, lda, B, ldb, batch, c1, nullptr, s)) != cudaSuccess) return e;
    TrsmConfig c2 = choose_trsm(0, 0, 1, 1, n, nrhs, batch);
    if ((e = launch_dtrsm(0, 0, 1, 1, n, nrhs, 1.0, A, lda, B, ldb, batch, c2, nullptr, s)) != cudaSuccess) return e;
    laswp_kernel<<<blocks, 256, 0, s>>>(n, nrhs, B, ldb, ipiv, sipiv, 1, batch);
    count_launch();
    return cudaGetLastError();
}

}  // namespace bf
