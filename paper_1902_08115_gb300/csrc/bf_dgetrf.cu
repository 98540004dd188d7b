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
#include <atomic>

#include "bf_internal.h"
#include "bf_lane.cuh"

namespace bf {

struct GetrfParams {
    int m, n;  // rows, columns (the lane form: m == n)
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

// ------------------------------------------------------------------ one problem per CTA
// For batches too small to fill the GPU one problem per thread, and for every m x n problem
// with m != n: right-looking by 16-column panels over the first min(m, n) columns, the panel in
// shared memory (W(i, c) = W[i + c m], rows J..m-1).  Per panel:
//   (1) the panel factored column by column: the pivot (first row of largest |a| below the
//       diagonal, taken only when strictly larger than |a_cc| -- a NaN never counts as larger),
//       the row interchange inside the panel, scaling by the pivot's reciprocal, and the
//       rank-1 update of the panel's later columns -- the steps, order and operations of the
//       lane form, so pivots agree with it;
//   (2) the panel back to global memory, and its interchanges applied to every other column
//       (one thread per column, the interchanges in order);
//   (3) U12 = L11^{-1} A12 (unit lower, one thread per column) and the trailing update
//       A22 -= L21 U12 on 4x4 register tiles.
// A wide problem (m < n) ends with U12 of its last panel (no rows left below); a tall one
// (m > n) ends with its last panel (no columns left to the right), L being m x n.
#define BF_GETRF_NB 16

__device__ __forceinline__ void argmax_pair(double& v, int& i, double v2, int i2) {
    if (v2 > v || (v2 == v && i2 < i)) {
        v = v2;
        i = i2;
    }
}

__global__ void __launch_bounds__(128, 4) dgetrf_cta_kernel(GetrfParams p) {
    extern __shared__ __align__(16) double sm_lu[];
    __shared__ double s_v[4];
    __shared__ int s_i[4];
    __shared__ int s_piv[BF_GETRF_NB];
    __shared__ int s_info;
    const int M = p.m, n = p.n, K = M < n ? M : n, lda = p.lda, T = blockDim.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    double* W = sm_lu;
    for (long long q = blockIdx.x; q < p.batch; q += gridDim.x) {
        double* A = p.A.mptr(q);
        int* piv = p.ipiv + q * p.sipiv;
        if (tid == 0) s_info = 0;
        for (int J = 0; J < K; J += BF_GETRF_NB) {
            const int nb = imin(BF_GETRF_NB, K - J), m = M - J;  // panel width, height
            for (int e = tid; e < m * nb; e += T) {
                const int c = e / m, i = e - c * m;
                W[i + c * M] = A[J + i + (long long)(J + c) * lda];
            }
            __syncthreads();
            // (1) the panel
            for (int c = 0; c < nb; c++) {
                double bv = -1.0;  // no candidate below the diagonal yet
                int bi = c;
                for (int i = c + 1 + tid; i < m; i += T) {
                    const double v = fabs(W[i + c * M]);
                    if (v > bv) {  // strictly larger: the first of equal maxima stays, NaN never wins
                        bv = v;
                        bi = i;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
                    const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
                    argmax_pair(bv, bi, v2, i2);
                }
                if (lane == 0) {
                    s_v[warp] = bv;
                    s_i[warp] = bi;
                }
                __syncthreads();
                if (tid == 0) {
                    for (int w = 1; w < (T >> 5); w++) argmax_pair(bv, bi, s_v[w], s_i[w]);
                    const int pr = (bv > fabs(W[c + c * M])) ? bi : c;
                    s_piv[c] = pr;
                    piv[J + c] = J + pr + 1;
                    if (W[pr + c * M] == 0.0 && s_info == 0) s_info = J + c + 1;
                }
                __syncthreads();
                const int pr = s_piv[c];
                if (pr != c) {
                    for (int c2 = tid; c2 < nb; c2 += T) {
                        const double t = W[c + c2 * M];
                        W[c + c2 * M] = W[pr + c2 * M];
                        W[pr + c2 * M] = t;
                    }
                    __syncthreads();
                }
                const double pv = W[c + c * M];
                if (pv != 0.0) {
                    const double rcp = 1.0 / pv;
                    for (int i = c + 1 + tid; i < m; i += T) W[i + c * M] *= rcp;
                    __syncthreads();
                }
                const int w2 = nb - c - 1, h = m - c - 1;
                for (int e = tid; e < w2 * h; e += T) {
                    const int c2 = c + 1 + e / h, i = c + 1 + e % h;
                    W[i + c2 * M] = fma(-W[i + c * M], W[c + c2 * M], W[i + c2 * M]);
                }
                __syncthreads();
            }
            // (2) the panel back, its interchanges on the other columns
            for (int e = tid; e < m * nb; e += T) {
                const int c = e / m, i = e - c * m;
                A[J + i + (long long)(J + c) * lda] = W[i + c * M];
            }
            for (int j = tid; j < n; j += T) {
                if (j >= J && j < J + nb) continue;
                double* col = A + (long long)j * lda;
                for (int c = 0; c < nb; c++) {
                    const int pr = J + s_piv[c];
                    if (pr != J + c) {
                        const double t = col[J + c];
                        col[J + c] = col[pr];
                        col[pr] = t;
                    }
                }
            }
            __syncthreads();
            if (J + nb < n) {
                // (3) U12 = L11^{-1} A12, then A22 -= L21 U12
                for (int j = J + nb + tid; j < n; j += T) {
                    double* col = A + (long long)j * lda + J;
                    double u[BF_GETRF_NB];
#pragma unroll
                    for (int c = 0; c < BF_GETRF_NB; c++) u[c] = c < nb ? col[c] : 0.0;
#pragma unroll
                    for (int c = 1; c < BF_GETRF_NB; c++) {
                        if (c >= nb) break;  // W holds nb <= M rows of L11: no read past them
#pragma unroll
                        for (int c2 = 0; c2 < c; c2++) u[c] = fma(-W[c + c2 * M], u[c2], u[c]);
                    }
#pragma unroll
                    for (int c = 0; c < BF_GETRF_NB; c++)
                        if (c < nb) col[c] = u[c];
                }
                __syncthreads();
                const int r = M - J - nb, tr = (r + 3) / 4;          // rows below the panel
                const int rc = n - J - nb, tc = (rc + 3) / 4;        // columns right of it
                for (int t = tid; t < tr * tc; t += T) {
                    const int i0 = 4 * (t % tr), j0 = 4 * (t / tr);  // rows / columns from J + nb
                    double acc[4][4];
#pragma unroll
                    for (int a = 0; a < 4; a++)
#pragma unroll
                        for (int b = 0; b < 4; b++) acc[a][b] = 0.0;
                    for (int c = 0; c < nb; c++) {
                        double l[4], u[4];
#pragma unroll
                        for (int a = 0; a < 4; a++) l[a] = W[nb + imin(i0 + a, r - 1) + c * M];
#pragma unroll
                        for (int b = 0; b < 4; b++) u[b] = A[J + c + (long long)(J + nb + imin(j0 + b, rc - 1)) * lda];
#pragma unroll
                        for (int a = 0; a < 4; a++)
#pragma unroll
                            for (int b = 0; b < 4; b++) acc[a][b] = fma(l[a], u[b], acc[a][b]);
                    }
#pragma unroll
                    for (int b = 0; b < 4; b++) {
                        if (j0 + b >= rc) continue;
                        double* col = A + (long long)(J + nb + j0 + b) * lda + J + nb;
#pragma unroll
                        for (int a = 0; a < 4; a++)
                            if (i0 + a < r) col[i0 + a] -= acc[a][b];
                    }
                }
                __syncthreads();
            }
        }
        if (tid == 0 && p.info) p.info[q] = s_info;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ four lanes per problem, in shared memory
// For orders up to kGetrfTeamMaxN.  The lane form above keeps each problem in global memory and
// its pivoting steps (the search down a column, the interchange of two whole rows, the scale)
// are one scattered access per lane per element: at n = 16 about 1,000 such accesses per problem
// against 1,365 multiply-adds, which bounds it by the L1 request rate.  Here a warp stages eight
// problems into shared memory with coalesced loads and factors each with a team of four lanes,
// right-looking, column by column (section 3.1 "dgetrf": the unblocked recurrence):
//   pivot    the first row of largest |a_ik|, i >= k (a NaN never counts as larger; a NaN in the
//            diagonal itself keeps row k), found on the magnitudes' bit patterns (integer
//            compares, no FP64 instruction) and reduced over the team with two shuffles
//   swap     rows k and p across all n columns, four columns per lane (when the pivot is not 0)
//   scale    l_ik = a_ik * (1 / a_kk) for i > k (when the pivot is not 0; else info = k + 1)
//   update   a_ij -= l_ik a_kj for i, j > k, lane r taking rows k+1+r, k+5+r, ...
// The operations on every element, and their order, are those of the lane form's column steps,
// so a problem gets the same pivots.  Storage: problem t of a warp at W + t PS, a(i, j) at
// i + j (n + 1); the odd column stride spreads a lane's four columns of a swap over four banks,
// and PS = 4 (mod 16) doubles puts the four problems of a half-warp on distinct banks.
// One instruction serves the warp's eight problems: a column step costs the warp one reciprocal,
// ceil(m/4) multiplies and ceil(m/4) m multiply-adds (m = n-1-k), with every lane of a team busy
// while its rows last.
__host__ __device__ inline int getrf_team_ps(int n) {
    const int ps = n * (n + 1);
    return ps + ((4 - ps % 16) + 16) % 16;
}

__global__ void __launch_bounds__(64) dgetrf_team_kernel(GetrfParams p) {
    extern __shared__ double getrf_sm[];
    const int n = p.n, ls = n + 1, PS = getrf_team_ps(n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t = lane >> 2, r = lane & 3;
    const long long q0 = ((long long)blockIdx.x * (blockDim.x >> 5) + warp) * 8;
    if (q0 >= p.batch) return;  // whole warps
    const int nq = (int)(p.batch - q0 < 8 ? p.batch - q0 : 8);
    double* W = getrf_sm + (size_t)warp * 8 * PS;
    // copy in: element e = (problem u, column j, row i), rows fastest, as asynchronous copies
    // straight into shared memory, all of a lane's in flight at once (no register staging)
    const int NE = 8 * n * n;
    const int dj = 32 / n, di = 32 - dj * n;
    {
        int u = 0, j = lane / n, i = lane - (lane / n) * n;
        while (j >= n) {
            j -= n;
            u++;
        }
        for (int e = lane; e < NE; e += 32) {
            if (u < nq) {
                const unsigned sa = (unsigned)__cvta_generic_to_shared(W + u * PS + i + j * ls);
                const double* ga = p.A.ptr(q0 + u) + i + (long long)j * p.lda;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(ga) : "memory");
            }
            i += di;
            j += dj;
            if (i >= n) {
                i -= n;
                j++;
            }
            while (j >= n) {
                j -= n;
                u++;
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    __syncwarp();
    double* Ap = W + t * PS;  // this team's problem
    int info = 0;
    for (int k = 0; k < n; k++) {
        const double* ck = Ap + k * ls;
        long long best = -2;
        int bi = k;
        for (int i = k + r; i < n; i += 4) {
            long long key = __double_as_longlong(ck[i]) & 0x7fffffffffffffffll;
            if (key > 0x7ff0000000000000ll) key = (i == k) ? 0x7fffffffffffffffll : -1;  // NaN
            if (key > best) {
                best = key;
                bi = i;
            }
        }
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
            const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (r == 0 && t < nq) p.ipiv[(q0 + t) * p.sipiv + k] = bi + 1;
        const double pv = ck[bi];
        const double rcp = __drcp_rn(pv);  // 1 / pv rounded to nearest, as the division; its latency
                                           // overlaps the interchange
        __syncwarp();
        if (pv != 0.0 && bi != k) {
            for (int j = r; j < n; j += 4) {
                const double a = Ap[k + j * ls], b = Ap[bi + j * ls];
                Ap[k + j * ls] = b;
                Ap[bi + j * ls] = a;
            }
        }
        if (pv == 0.0 && info == 0) info = k + 1;
        __syncwarp();
        // rows k+1+4h+r: the groups of four rows that exist for the warp's first lane are taken
        // (a warp-uniform test), so no FP64 instruction is issued for a group without rows (a
        // masked FP64 lane costs a full one); within a group, lanes past n sit out
#pragma unroll
        for (int h = 0; h < 4; h++) {
            if (k + 1 + 4 * h >= n) break;
            const int i = k + 1 + 4 * h + r;
            const bool act = i < n;
            double l = act ? Ap[i + k * ls] : 0.0;
            if (act && pv != 0.0) {
                l *= rcp;
                Ap[i + k * ls] = l;
            }
            for (int j = k + 1; j < n; j++) {
                double* cj = Ap + j * ls;
                const double ukj = cj[k];
                if (act) cj[i] = fma(-l, ukj, cj[i]);
            }
        }
        __syncwarp();
    }
    if (r == 0 && t < nq && p.info) p.info[q0 + t] = info;
    // copy out
    {
        int u = 0, j = lane / n, i = lane - (lane / n) * n;
        while (j >= n) {
            j -= n;
            u++;
        }
        for (int e = lane; e < NE; e += 32) {
            if (u < nq) p.A.mptr(q0 + u)[i + (long long)j * p.lda] = W[u * PS + i + j * ls];
            i += di;
            j += dj;
            if (i >= n) {
                i -= n;
                j++;
            }
            while (j >= n) {
                j -= n;
                u++;
            }
        }
    }
}

cudaError_t launch_dgetrf(int m, int n, MatRef A, int lda, int* ipiv, long long sipiv, int* info, long long batch,
                          cudaStream_t s) {
    if (batch == 0) return cudaSuccess;
    if (m == 0 || n == 0) return info ? cudaMemsetAsync(info, 0, sizeof(int) * (size_t)batch, s) : cudaSuccess;
    GetrfParams p;
    p.m = m; p.n = n; p.A = A; p.lda = lda; p.ipiv = ipiv; p.sipiv = sipiv; p.batch = batch; p.info = info;
    if (m != n || choose_getrf(n, batch) == VAR_CTA) {
        const size_t smem = sizeof(double) * (size_t)BF_GETRF_NB * m;
        // the dynamic limit is raised once to the largest panel (kGetrfMaxRows rows): the kernel's
        // static shared memory comes on top, so a panel of exactly 48 KB (m = 384) needs it too
        static std::atomic<int> raised{0};
        if (!raised.load(std::memory_order_acquire)) {
            const cudaError_t e = cudaFuncSetAttribute(dgetrf_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)(sizeof(double) * BF_GETRF_NB * kGetrfMaxRows));
            if (e != cudaSuccess) return e;
            raised.store(1, std::memory_order_release);
        }
        const long long cap = kSMs * 16;
        dgetrf_cta_kernel<<<(unsigned)(batch < cap ? batch : cap), 128, smem, s>>>(p);
        count_launch();
        return cudaGetLastError();
    }
    if (choose_getrf(n, batch) == VAR_TEAM) {  // n <= kGetrfTeamMaxN: 16 problems per 64-thread CTA
        const size_t smem = sizeof(double) * 16 * (size_t)getrf_team_ps(n);
        dgetrf_team_kernel<<<(unsigned)((batch + 15) / 16), 64, smem, s>>>(p);
        count_launch();
        return cudaGetLastError();
    }
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
