// bf_backward.cu -- hand-written reverse-mode (adjoint) routines for the
// batched dgemm, dtrsm and dpotrf, built from this library's kernels.
//
// dgemm, C = alpha op(A) op(B) + beta C0 (section 2.1):
//   Abar = alpha Cbar op(B)^T (transposed when op(A) = A^T),
//   Bbar = alpha op(A)^T Cbar (transposed when op(B) = B^T),  C0bar = beta Cbar.
// dtrsm, op(A) X = alpha B (left) / X op(A) = alpha B (right) (section 3.1):
//   Z solves op(A)^T Z = Xbar (left) / Z op(A)^T = Xbar (right);
//   Bbar = alpha Z;  op(A)bar = -Z X^T (left) / -X^T Z (right), kept on the
//   stored triangle of A (without the diagonal when it is unit).
// dpotrf, A = L L^T (section 3.1 "dpotrf"), the symmetric form published by
// I. Murray ("Differentiation of the Cholesky decomposition", 2016):
//   P = Phi(L^T Lbar)  (lower triangle, diagonal halved),
//   S = L^{-T} P L^{-1}  (two triangular solves),  Abar = (S + S^T) / 2.
//   Derivation: dA = dL L^T + L dL^T gives L^{-1} dL = Phi(L^{-1} dA L^{-T}),
//   and Phi is self-adjoint, so <Lbar, dL> = <L^{-T} Phi(L^T Lbar) L^{-1}, dA>.
#include "bf_internal.h"
#include "../../include/bfgpu.h"

namespace bf {

// P = Phi(L^T Lbar) for every problem, written to the full n x n of `out` (upper part zero).
// One thread per (lower 4x4 tile, problem), problem index fastest: the 32 lanes of a warp
// work on the same tile of 32 problems, so every lane runs the same k-loop length.  upper: L and
// Lbar are read as the transposes of the upper triangles stored (A = U^T U: L = U^T).
__global__ void __launch_bounds__(256)
phi_ltlbar_kernel(int n, MatRef L, int ldl, MatRef Lb, int ldlb, MatRef O, int ldo, long long batch, int nt,
                  int upper) {
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long ntile = (long long)nt * (nt + 1) / 2;
    if (gt >= ntile * batch) return;
    const long long q = gt % batch;
    const int t = (int)(gt / batch);
    int I = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while ((I + 1) * (I + 2) / 2 <= t) I++;
    while (I * (I + 1) / 2 > t) I--;
    const int J = t - I * (I + 1) / 2;
    const int i0 = 4 * I, j0 = 4 * J;
    const double* l = L.ptr(q);
    const double* lb = Lb.ptr(q);
    double* o = O.mptr(q);
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] = 0.0;
    // P_ij = sum_{k >= i} L(k, i) Lbar(k, j) for i >= j; structural zeros masked.  Lower storage
    // with both operands 16-byte aligned at even rows: k in pairs, L(k, i) and L(k+1, i) one
    // 16-byte load (i0 is a multiple of 4, so every pair starts on an even row)
    int k = i0;
    if (!upper && ((reinterpret_cast<uintptr_t>(l) | reinterpret_cast<uintptr_t>(lb)) & 15u) == 0 &&
        ((ldl | ldlb) & 1) == 0) {
        for (; k + 1 < n; k += 2) {
            double2 lp[4], bp[4];
#pragma unroll
            for (int a = 0; a < 4; a++)
                lp[a] = *reinterpret_cast<const double2*>(l + k + (long long)imin(i0 + a, n - 1) * ldl);
#pragma unroll
            for (int b = 0; b < 4; b++)
                bp[b] = *reinterpret_cast<const double2*>(lb + k + (long long)imin(j0 + b, n - 1) * ldlb);
#pragma unroll
            for (int h = 0; h < 2; h++) {
                double li[4], lbj[4];
#pragma unroll
                for (int a = 0; a < 4; a++) {
                    const int i = i0 + a;
                    li[a] = (i < n && k + h >= i) ? (h ? lp[a].y : lp[a].x) : 0.0;
                }
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    const int j = j0 + b;
                    lbj[b] = (j < n && k + h >= j) ? (h ? bp[b].y : bp[b].x) : 0.0;
                }
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int b = 0; b < 4; b++) acc[a][b] = fma(li[a], lbj[b], acc[a][b]);
            }
        }
    }
    for (; k < n; k++) {
        double li[4], lbj[4];
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int i = i0 + a;
            li[a] = (i < n && k >= i) ? l[upper ? i + (long long)k * ldl : k + (long long)i * ldl] : 0.0;
        }
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const int j = j0 + b;
            lbj[b] = (j < n && k >= j) ? lb[upper ? j + (long long)k * ldlb : k + (long long)j * ldlb] : 0.0;
        }
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++) acc[a][b] = fma(li[a], lbj[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; a++) {
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const int i = i0 + a, j = j0 + b;
            if (i >= n || j >= n) continue;
            if (i > j) {
                o[i + (long long)j * ldo] = acc[a][b];
                o[j + (long long)i * ldo] = 0.0;
            } else if (i == j) {
                o[i + (long long)j * ldo] = 0.5 * acc[a][b];
            } else {
                o[i + (long long)j * ldo] = 0.0;  // strict upper part of a diagonal tile
            }
        }
    }
}

// G = (S + S^T) / 2 in place: one CTA of 32 x 8 threads per (problem, pair of 32 x 32 tiles
// (bi, bj), bi >= bj).  Both tiles are read coalesced (consecutive threads, consecutive rows)
// into shared memory, averaged with the transpose there, and written back coalesced; a diagonal
// tile pairs with itself.  The same value goes to (i, j) and (j, i), so G is exactly symmetric.
__global__ void __launch_bounds__(256) symmetrize_kernel(int n, MatRef S, int lds, long long batch, int nt) {
    __shared__ double ta[32][33], tb[32][33];
    const long long pairs = (long long)nt * (nt + 1) / 2;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (long long w = blockIdx.x; w < pairs * batch; w += gridDim.x) {
        const long long q = w / pairs;
        const int t = (int)(w - q * pairs);
        int bi = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
        while ((bi + 1) * (bi + 2) / 2 <= t) bi++;
        while (bi * (bi + 1) / 2 > t) bi--;
        const int bj = t - bi * (bi + 1) / 2;
        double* s = S.mptr(q);
        const int r0 = 32 * bi, c0 = 32 * bj;  // tile A: rows r0.., columns c0..; tile B its mirror
        __syncthreads();
        for (int c = ty; c < 32; c += 8) {
            const int i = r0 + tx, j = c0 + c;
            ta[c][tx] = (i < n && j < n) ? s[i + (long long)j * lds] : 0.0;  // ta[c][r] = A(r0+r, c0+c)
            const int i2 = c0 + tx, j2 = r0 + c;
            tb[c][tx] = (i2 < n && j2 < n) ? s[i2 + (long long)j2 * lds] : 0.0;  // tb[c][r] = S(c0+r, r0+c)
        }
        __syncthreads();
        for (int c = ty; c < 32; c += 8) {
            // A(r0+tx, c0+c) and its mirror S(c0+c, r0+tx) = tb[tx][c]
            const double g = 0.5 * (ta[c][tx] + tb[tx][c]);
            const int i = r0 + tx, j = c0 + c;
            if (i < n && j < n) s[i + (long long)j * lds] = g;
        }
        __syncthreads();
        if (bi != bj) {
            for (int c = ty; c < 32; c += 8) {
                // S(c0+tx, r0+c) = the average of A(r0+c, c0+tx) and itself's mirror
                const double g = 0.5 * (tb[c][tx] + ta[tx][c]);
                const int i = c0 + tx, j = r0 + c;
                if (i < n && j < n) s[i + (long long)j * lds] = g;
            }
        }
    }
}

// Y = beta X (X and Y m x n, may alias)
__global__ void __launch_bounds__(256)
dscal_copy_kernel(int m, int n, double beta, MatRef X, int ldx, MatRef Y, int ldy, long long batch) {
    const long long per = (long long)m * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per * batch;
         e += (long long)gridDim.x * blockDim.x) {
        const long long q = e / per;
        const long long r = e - q * per;
        const int j = (int)(r / m), i = (int)(r - (long long)j * m);
        const double v = X.ptr(q)[i + (long long)j * ldx];
        Y.mptr(q)[i + (long long)j * ldy] = beta * v;
    }
}

static cudaError_t launch_scal_copy(int m, int n, double beta, MatRef X, int ldx, MatRef Y, int ldy,
                                    long long batch, cudaStream_t s) {
    if (m == 0 || n == 0 || batch == 0) return cudaSuccess;
    long long total = (long long)m * n * batch;
    long long blocks = (total + 255) / 256;
    if (blocks > kSMs * 64) blocks = kSMs * 64;
    dscal_copy_kernel<<<(unsigned)blocks, 256, 0, s>>>(m, n, beta, X, ldx, Y, ldy, batch);
    count_launch();
    return cudaGetLastError();
}

// Tidy a factored batch: the strict triangle opposite the factor (upper = 0: the strict upper
// one) is set to zero, and every entry of the n x n of a problem whose info is nonzero is set to
// NaN, so that a failed factorisation cannot pass on as a finite factor.  Element index fastest
// within a problem (consecutive threads, consecutive rows of a column: coalesced).
__global__ void __launch_bounds__(256)
dtrfill_kernel(int n, int upper, double* A, int lda, long long stride, const int* info, long long batch) {
    const long long per = (long long)n * n;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per * batch;
         e += (long long)gridDim.x * blockDim.x) {
        const long long q = e / per;
        const long long r = e - q * per;
        const int j = (int)(r / n), i = (int)(r - (long long)j * n);
        double* a = A + q * stride + i + (long long)j * lda;
        if (info && info[q] != 0) {
            *a = nan;
        } else if (upper ? i > j : i < j) {
            *a = 0.0;
        }
    }
}

// For n <= 32 the whole Cholesky adjoint in one kernel, one warp per problem.  L (the view's lower
// factor: with UP the transpose of the stored upper triangle), Lbar (likewise) and the
// reciprocal diagonal of L sit in shared memory.
//   (0) P = Phi(L^T Lbar).  The 528 entries (i, j), i >= j, of the lower triangle are dealt to
//       the lanes in row order (entry e = i (i + 1) / 2 + j: lane e % 32, register e / 32).  Step
//       k adds L(k, i) Lbar(k, j) to every entry with i <= k, which are the first
//       (k + 1)(k + 2) / 2 entries, so a step issues ceil((k + 1)(k + 2) / 64) multiply-adds
//       with at most one of them partly masked: 203 warp instructions at n = 32 for 5,984 lane
//       multiply-adds (187 full warps' worth).  Each entry adds its nonzero terms in increasing
//       k, as the tile kernel of larger orders does, so P is the same; the diagonal is halved.
//   (1) lane c holds column c of P and back-substitutes it against L^T: for j = n-1 .. 0,
//       x_j *= 1 / L(j, j), then x_i -= L(j, i) x_j for i < j -- every lane reads the same
//       L(j, i) (a broadcast) and updates its own column, all 32 lanes busy;
//   (2) the columns of S1 go through shared memory to rows (lane r: row r of S1), and each row
//       is solved against L the same way (S L = S1 is back substitution on the row);
//   (3) the rows of S go through shared memory once more, so lane r also holds column r, and
//       lane r writes row r of (S + S^T) / 2 -- consecutive lanes, consecutive rows: coalesced.
// The two halves of a symmetric pair are the same sum, so Abar is exactly symmetric.  Against
// the Phi tile kernel, two row-parallel dtrsm launches and the symmetrizing kernel, P, S1 and S
// never go to memory.
#define BF_ADJ_WARPS 2
template <bool UP>
__global__ void __launch_bounds__(32 * BF_ADJ_WARPS, 6)
chol_adjoint32_kernel(int n, MatRef L, int ldl, MatRef Lb, int ldlb, MatRef Ab, int ldab, long long batch) {
    __shared__ double sL[BF_ADJ_WARPS][32][33];  // sL[w][j][i] = L(i, j)
    __shared__ double sW[BF_ADJ_WARPS][32][33];  // column-major staging: sW[w][c][r] = M(r, c)
    __shared__ double sR[BF_ADJ_WARPS][32];      // 1 / L(j, j)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double(*Lw)[33] = sL[w];
    double(*Ww)[33] = sW[w];
    for (long long q = (long long)blockIdx.x * BF_ADJ_WARPS + w; q < batch; q += (long long)gridDim.x * BF_ADJ_WARPS) {
        const double* l = L.ptr(q);
        const double* lb = Lb.ptr(q);
        double* a = Ab.mptr(q);
        // L and Lbar (lower, zero above), column by column, rows by lane: coalesced
        for (int j = 0; j < n; j++) {
            double v = 0.0, vb = 0.0;
            if (lane < n && lane >= j) {
                v = UP ? l[j + (long long)lane * ldl] : l[lane + (long long)j * ldl];
                vb = UP ? lb[j + (long long)lane * ldlb] : lb[lane + (long long)j * ldlb];
            }
            Lw[j][lane] = v;
            Ww[j][lane] = vb;
        }
        __syncwarp();
        if (lane < n) sR[w][lane] = 1.0 / Lw[lane][lane];
        // (0) P = Phi(L^T Lbar), this lane's entries of the lower triangle
        {
            int ie[17], je[17];
#pragma unroll
            for (int r = 0; r < 17; r++) {
                const int e = 32 * r + lane;
                int i = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
                if ((i + 1) * (i + 2) / 2 <= e) i++;
                if (i * (i + 1) / 2 > e) i--;
                ie[r] = e < 528 ? i : 31;  // past the triangle: never active, never stored
                je[r] = e < 528 ? e - i * (i + 1) / 2 : 0;
            }
            double acc[17];
#pragma unroll
            for (int r = 0; r < 17; r++) acc[r] = 0.0;
            for (int k = 0; k < n; k++) {
                const int tk = (k + 1) * (k + 2) / 2;  // entries with i <= k
#pragma unroll
                for (int r = 0; r < 17; r++) {
                    if (32 * r >= tk) break;
                    if (32 * r + lane < tk) acc[r] = fma(Lw[ie[r]][k], Ww[je[r]][k], acc[r]);
                }
            }
            __syncwarp();  // every lane is done with Lbar
#pragma unroll
            for (int r = 0; r < 17; r++)
                if (32 * r + lane < 528) Ww[je[r]][ie[r]] = ie[r] == je[r] ? 0.5 * acc[r] : acc[r];  // P(i, j)
        }
        __syncwarp();
        double x[32];
#pragma unroll
        for (int i = 0; i < 32; i++) x[i] = i >= lane ? Ww[lane][i] : 0.0;  // column `lane` of P
        __syncwarp();
        // (1) S1 = L^{-T} P, column `lane`
#pragma unroll
        for (int j = 31; j >= 0; j--) {
            if (j < n) {
                x[j] *= sR[w][j];
#pragma unroll
                for (int i = 0; i < j; i++) x[i] = fma(-Lw[i][j], x[j], x[i]);
            }
        }
        // (2) rows of S1, then S = S1 L^{-1}, row `lane`
#pragma unroll
        for (int i = 0; i < 32; i++) Ww[lane][i] = x[i];  // sW[c = lane][r = i] = S1(i, lane)
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 32; j++) x[j] = Ww[j][lane];  // S1(lane, j)
        __syncwarp();
#pragma unroll
        for (int j = 31; j >= 0; j--) {
            if (j < n) {
                x[j] *= sR[w][j];
#pragma unroll
                for (int i = 0; i < j; i++) x[i] = fma(-Lw[i][j], x[j], x[i]);
            }
        }
        // (3) column `lane` of S beside its row, and row `lane` of (S + S^T) / 2 out
#pragma unroll
        for (int j = 0; j < 32; j++) Ww[j][lane] = x[j];  // sW[c = j][r = lane] = S(lane, j)
        __syncwarp();
        if (lane < n) {
#pragma unroll
            for (int i = 0; i < 32; i++)
                if (i < n) a[lane + (long long)i * ldab] = 0.5 * (x[i] + Ww[lane][i]);  // (S(lane,i) + S(i,lane)) / 2
        }
        __syncwarp();
    }
}

cudaError_t launch_dpotrf_backward(int n, MatRef L, int ldl, MatRef Lb, int ldlb, MatRef Ab, int ldab,
                                   long long batch, cudaStream_t s, int upper) {
    if (n == 0 || batch == 0) return cudaSuccess;
    const int nt = (n + 3) / 4;
    long long threads = (long long)nt * (nt + 1) / 2 * batch;
    if (n <= 32) {  // Phi, the solves and the symmetrizing in one kernel
        const long long blocks = (batch + BF_ADJ_WARPS - 1) / BF_ADJ_WARPS;
        if (upper)
            chol_adjoint32_kernel<true><<<(unsigned)blocks, 32 * BF_ADJ_WARPS, 0, s>>>(n, L, ldl, Lb, ldlb, Ab, ldab,
                                                                                      batch);
        else
            chol_adjoint32_kernel<false><<<(unsigned)blocks, 32 * BF_ADJ_WARPS, 0, s>>>(n, L, ldl, Lb, ldlb, Ab, ldab,
                                                                                       batch);
        count_launch();
        return cudaGetLastError();
    }
    phi_ltlbar_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(n, L, ldl, Lb, ldlb, Ab, ldab, batch, nt,
                                                                         upper);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // S1 = L^{-T} P (left, lower, transposed), then S = S1 L^{-1} (right, lower, not transposed);
    // upper (L = U^T): S1 = U^{-1} P (left, upper), then S = S1 U^{-T} (right, upper, transposed)
    const int tr1 = upper ? 0 : 1, tr2 = upper ? 1 : 0;
    TrsmConfig c1 = choose_trsm(0, upper, tr1, 0, n, n, batch);
    e = launch_dtrsm(0, upper, tr1, 0, n, n, 1.0, L, ldl, Ab, ldab, batch, c1, nullptr, s);
    if (e != cudaSuccess) return e;
    TrsmConfig c2 = choose_trsm(1, upper, tr2, 0, n, n, batch);
    e = launch_dtrsm(1, upper, tr2, 0, n, n, 1.0, L, ldl, Ab, ldab, batch, c2, nullptr, s);
    if (e != cudaSuccess) return e;
    if (n > 1) {
        const int ntile = (n + 31) / 32;
        const long long work = (long long)ntile * (ntile + 1) / 2 * batch;
        const long long grid = work < kSMs * 16 ? work : kSMs * 16;
        symmetrize_kernel<<<(unsigned)grid, 256, 0, s>>>(n, Ab, ldab, batch, ntile);
        count_launch();
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace bf

using namespace bf;

static inline bool cis_n(char c) { return c == 'N' || c == 'n'; }
static inline bool cis_t(char c) { return c == 'T' || c == 't' || c == 'C' || c == 'c'; }
static inline bool cis_l(char c) { return c == 'L' || c == 'l'; }
static inline bool cis_u(char c) { return c == 'U' || c == 'u'; }
static inline bool cis_r(char c) { return c == 'R' || c == 'r'; }
static inline int cmax1(int a) { return a > 1 ? a : 1; }
static inline int cstat(cudaError_t e) { return e == cudaSuccess ? BF_SUCCESS : BF_ERR_CUDA; }

extern "C" int bf_dgemm_backward_strided_batched(
    char transa, char transb, int m, int n, int k, double alpha, const double* A, int lda, long long strideA,
    const double* B, int ldb, long long strideB, double beta, const double* Cbar, int ldcb, long long strideCbar,
    double* Abar, int ldab, long long strideAbar, double* Bbar, int ldbb, long long strideBbar, double* C0bar,
    int ldc0b, long long strideC0bar, int batch, bf_stream_t stream) {
    if (!(cis_n(transa) || cis_t(transa))) return -1;
    if (!(cis_n(transb) || cis_t(transb))) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 0) return -5;
    const bool ta = cis_t(transa), tb = cis_t(transb);
    const int rA = ta ? k : m, cA = ta ? m : k, rB = tb ? n : k, cB = tb ? k : n;
    if (lda < cmax1(rA)) return -8;
    if (ldb < cmax1(rB)) return -11;
    if (ldcb < cmax1(m)) return -15;
    if (Abar && ldab < cmax1(rA)) return -18;
    if (Bbar && ldbb < cmax1(rB)) return -21;
    if (C0bar && ldc0b < cmax1(m)) return -24;
    if (batch < 0) return -26;
    const bool work = batch > 0;
    if (work && Abar && n > 0 && cA > 0 && !B) return -10;
    if (work && Bbar && m > 0 && cB > 0 && !A) return -7;
    if (work && (Abar || Bbar || C0bar) && !Cbar) return -14;
    if (!work) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    MatRef mA = mat_strided(A, strideA), mB = mat_strided(B, strideB), mC = mat_strided(Cbar, strideCbar);
    cudaError_t e = cudaSuccess;
    if (Abar && rA > 0 && cA > 0) {
        MatRef o = mat_strided(Abar, strideAbar);
        if (!ta) {  // Abar (m x k) = alpha Cbar op(B)^T
            GemmConfig c = choose_gemm(false, !tb, m, k, n, ldcb, batch);
            e = launch_dgemm(false, !tb, m, k, n, alpha, mC, ldcb, mB, ldb, 0.0, o, ldab, batch, c, 0, nullptr, s);
        } else {  // Abar (k x m) = alpha op(B) Cbar^T
            GemmConfig c = choose_gemm(tb, true, k, m, n, ldb, batch);
            e = launch_dgemm(tb, true, k, m, n, alpha, mB, ldb, mC, ldcb, 0.0, o, ldab, batch, c, 0, nullptr, s);
        }
        if (e != cudaSuccess) return cstat(e);
    }
    if (Bbar && rB > 0 && cB > 0) {
        MatRef o = mat_strided(Bbar, strideBbar);
        if (!tb) {  // Bbar (k x n) = alpha op(A)^T Cbar
            GemmConfig c = choose_gemm(!ta, false, k, n, m, lda, batch);
            e = launch_dgemm(!ta, false, k, n, m, alpha, mA, lda, mC, ldcb, 0.0, o, ldbb, batch, c, 0, nullptr, s);
        } else {  // Bbar (n x k) = alpha Cbar^T op(A)
            GemmConfig c = choose_gemm(true, ta, n, k, m, ldcb, batch);
            e = launch_dgemm(true, ta, n, k, m, alpha, mC, ldcb, mA, lda, 0.0, o, ldbb, batch, c, 0, nullptr, s);
        }
        if (e != cudaSuccess) return cstat(e);
    }
    if (C0bar && m > 0 && n > 0)
        e = launch_scal_copy(m, n, beta, mC, ldcb, mat_strided(C0bar, strideC0bar), ldc0b, batch, s);
    return cstat(e);
}

// A triangle-masked product (the dtrsm adjoint's op(A)bar on the stored triangle) skips only
// whole super-tiles: the size switch's square super-tile (32 x 32 at order 32) covers the
// diagonal and skips nothing.  8 x 8 super-tiles (4 threads of 4 x 4 tiles each) let the mask
// drop the 6 of 16 wholly off the triangle at order 32, 28 of 64 at order 64.
static GemmConfig tri_config(GemmConfig c, int m) {
    if (c.variant == VAR_DIRECT && m > 8) {
        c.TM = c.TN = 8;
        c.P = 64;  // 4 threads per problem: 256-thread CTAs
    }
    return c;
}

extern "C" int bf_dtrsm_backward_strided_batched(char side, char uplo, char transa, char diag, int m, int n,
                                                 double alpha, const double* A, int lda, long long strideA,
                                                 const double* X, int ldx, long long strideX, double* XBbar,
                                                 int ldxb, long long strideXB, double* Abar, int ldab,
                                                 long long strideAbar, int batch, bf_stream_t stream) {
    if (!(cis_l(side) || cis_r(side))) return -1;
    if (!(cis_l(uplo) || cis_u(uplo))) return -2;
    if (!(cis_n(transa) || cis_t(transa))) return -3;
    if (!(cis_u(diag) || cis_n(diag))) return -4;
    if (m < 0) return -5;
    if (n < 0) return -6;
    const bool left = cis_l(side);
    const int order = left ? m : n;
    if (lda < cmax1(order)) return -9;
    if (ldx < cmax1(m)) return -12;
    if (ldxb < cmax1(m)) return -15;
    if (Abar && ldab < cmax1(order)) return -18;
    if (batch < 0) return -20;
    if (alpha == 0.0) return -7;  // X does not depend on A, B: the adjoint is not defined by this formula
    const bool work = m > 0 && n > 0 && batch > 0;
    if (work && !A) return -8;
    if (work && Abar && !X) return -11;
    if (work && !XBbar) return -14;
    if (!work) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    const int sd = left ? 0 : 1, up = cis_u(uplo) ? 1 : 0, tr = cis_t(transa) ? 1 : 0, un = cis_u(diag) ? 1 : 0;
    MatRef mA = mat_strided(A, strideA), mX = mat_strided(X, strideX), mZ = mat_strided(XBbar, strideXB);
    // Z = op(A)^{-T} Xbar (left) or Xbar op(A)^{-T} (right), in place
    TrsmConfig tc = choose_trsm(sd, up, !tr, un, m, n, batch);
    cudaError_t e = launch_dtrsm(sd, up, !tr, un, m, n, 1.0, mA, lda, mZ, ldxb, batch, tc, nullptr, s);
    if (e != cudaSuccess) return cstat(e);
    if (Abar) {
        const int tri = up ? (un ? TRI_SUPPER : TRI_UPPER) : (un ? TRI_SLOWER : TRI_LOWER);
        MatRef o = mat_strided(Abar, strideAbar);
        if (left) {
            // op(A)bar = -Z X^T (m x m); Abar = op(A)bar or its transpose -X Z^T
            MatRef P = tr ? mX : mZ, Q = tr ? mZ : mX;
            const int ldp = tr ? ldx : ldxb, ldq = tr ? ldxb : ldx;
            GemmConfig c = tri_config(choose_gemm(false, true, m, m, n, ldp, batch), m);
            e = launch_dgemm(false, true, m, m, n, -1.0, P, ldp, Q, ldq, 0.0, o, ldab, batch, c, tri, nullptr, s);
        } else {
            // op(A)bar = -X^T Z (n x n); Abar = op(A)bar or its transpose -Z^T X
            MatRef P = tr ? mZ : mX, Q = tr ? mX : mZ;
            const int ldp = tr ? ldxb : ldx, ldq = tr ? ldx : ldxb;
            GemmConfig c = tri_config(choose_gemm(true, false, n, n, m, ldp, batch), n);
            e = launch_dgemm(true, false, n, n, m, -1.0, P, ldp, Q, ldq, 0.0, o, ldab, batch, c, tri, nullptr, s);
        }
        if (e != cudaSuccess) return cstat(e);
    }
    if (alpha != 1.0) e = launch_scal_copy(m, n, alpha, mZ, ldxb, mZ, ldxb, batch, s);
    return cstat(e);
}

extern "C" int bf_dpotrf_backward_strided_batched(char uplo, int n, const double* L, int ldl, long long strideL,
                                                  const double* Lbar, int ldlb, long long strideLbar, double* Abar,
                                                  int ldab, long long strideAbar, int batch, bf_stream_t stream) {
    if (!(cis_l(uplo) || cis_u(uplo))) return -1;
    if (n < 0) return -2;
    if (ldl < cmax1(n)) return -4;
    if (ldlb < cmax1(n)) return -7;
    if (ldab < cmax1(n)) return -10;
    if (batch < 0) return -12;
    if (batch > 1 && strideAbar < (long long)ldab * n) return -11;
    const bool work = n > 0 && batch > 0;
    if (work && !L) return -3;
    if (work && !Lbar) return -6;
    if (work && !Abar) return -9;
    if (!work) return 0;
    return cstat(launch_dpotrf_backward(n, mat_strided(L, strideL), ldl, mat_strided(Lbar, strideLbar), ldlb,
                                        mat_strided(Abar, strideAbar), ldab, batch, (cudaStream_t)stream,
                                        cis_u(uplo) ? 1 : 0));
}

// The dpotrs adjoint: the two triangular-solve adjoints of X = L^{-T} L^{-1} B with their
// triangle gradients summed in one buffer -- the first masked product writes its triangle, the
// second accumulates onto it (beta = 1), and the strict other triangle is set to zero.
extern "C" int bf_dpotrs_backward_strided_batched(char uplo, int n, int nrhs, const double* L, int ldl,
                                                  long long strideL, const double* X, int ldx, long long strideX,
                                                  const double* Y, int ldy, long long strideY, double* XBbar,
                                                  int ldxb, long long strideXB, double* Lbar, int ldlb,
                                                  long long strideLbar, int batch, bf_stream_t stream) {
    if (!(cis_l(uplo) || cis_u(uplo))) return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (ldl < cmax1(n)) return -5;
    if (ldx < cmax1(n)) return -8;
    if (ldy < cmax1(n)) return -11;
    if (ldxb < cmax1(n)) return -14;
    if (ldlb < cmax1(n)) return -17;
    if (batch < 0) return -19;
    if (batch > 1 && strideLbar < (long long)ldlb * n) return -18;
    const bool work = n > 0 && batch > 0;
    if (work && !L) return -4;
    if (work && !Lbar) return -16;
    if (work && nrhs > 0 && !X) return -7;
    if (work && nrhs > 0 && !Y) return -10;
    if (work && nrhs > 0 && !XBbar) return -13;
    if (!work) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    const int up = cis_u(uplo) ? 1 : 0;
    MatRef mL = mat_strided(L, strideL), mX = mat_strided(X, strideX), mY = mat_strided(Y, strideY);
    MatRef mZ = mat_strided(XBbar, strideXB), o = mat_strided(Lbar, strideLbar);
    const int tri = up ? TRI_UPPER : TRI_LOWER;
    cudaError_t e;
    if (nrhs == 0) {  // no right-hand sides: a zero gradient
        GemmConfig z{VAR_DIRECT, 4, 4, 0, 1};
        return cstat(launch_dgemm(false, false, n, n, 0, 0.0, o, ldlb, o, ldlb, 0.0, o, ldlb, batch, z, 0, nullptr, s));
    }
    // Z1: L Z1 = Xbar ('U': U^T Z1 = Xbar), in place -- the adjoint solve of X = op(L)^{-1} Y
    TrsmConfig t1 = choose_trsm(0, up, up, 0, n, nrhs, batch);
    if ((e = launch_dtrsm(0, up, up, 0, n, nrhs, 1.0, mL, ldl, mZ, ldxb, batch, t1, nullptr, s)) != cudaSuccess)
        return cstat(e);
    // Lbar = -X Z1^T on the lower triangle ('U': -Z1 X^T on the upper)
    {
        MatRef P = up ? mZ : mX, Q = up ? mX : mZ;
        const int ldp = up ? ldxb : ldx, ldq = up ? ldx : ldxb;
        GemmConfig c = tri_config(choose_gemm(false, true, n, n, nrhs, ldp, batch), n);
        if ((e = launch_dgemm(false, true, n, n, nrhs, -1.0, P, ldp, Q, ldq, 0.0, o, ldlb, batch, c, tri, nullptr,
                              s)) != cudaSuccess)
            return cstat(e);
    }
    // Z2: L^T Z2 = Z1 ('U': U Z2 = Z1), in place -- the adjoint solve of Y = op(L)^{-1} B
    TrsmConfig t2 = choose_trsm(0, up, !up, 0, n, nrhs, batch);
    if ((e = launch_dtrsm(0, up, !up, 0, n, nrhs, 1.0, mL, ldl, mZ, ldxb, batch, t2, nullptr, s)) != cudaSuccess)
        return cstat(e);
    // Lbar += -Z2 Y^T on the lower triangle ('U': -Y Z2^T on the upper)
    MatRef P = up ? mY : mZ, Q = up ? mZ : mY;
    const int ldp = up ? ldy : ldxb, ldq = up ? ldxb : ldy;
    GemmConfig c = tri_config(choose_gemm(false, true, n, n, nrhs, ldp, batch), n);
    if ((e = launch_dgemm(false, true, n, n, nrhs, -1.0, P, ldp, Q, ldq, 1.0, o, ldlb, batch, c, tri, nullptr, s)) !=
        cudaSuccess)
        return cstat(e);
    // zeros in the strict other triangle (a separate pass: a zero-writing branch in the product's
    // store measured 4-17 % slower on some plain dgemm shapes that share that kernel)
    const long long total = (long long)n * n * batch;
    long long blocks = (total + 255) / 256;
    if (blocks > kSMs * 32) blocks = kSMs * 32;
    dtrfill_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, up, Lbar, ldlb, strideLbar, nullptr, batch);
    count_launch();
    return cstat(cudaGetLastError());
}

extern "C" int bf_dtrfill_strided_batched(char uplo, int n, double* A, int lda, long long strideA, const int* info,
                                          int batch, bf_stream_t stream) {
    if (!(cis_l(uplo) || cis_u(uplo))) return -1;
    if (n < 0) return -2;
    if (lda < cmax1(n)) return -4;
    if (batch < 0) return -7;
    if (batch > 1 && strideA < (long long)lda * n) return -5;
    if (n == 0 || batch == 0) return 0;
    if (!A) return -3;
    const long long total = (long long)n * n * batch;
    long long blocks = (total + 255) / 256;
    if (blocks > kSMs * 32) blocks = kSMs * 32;
    dtrfill_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(n, cis_u(uplo) ? 1 : 0, A, lda, strideA, info,
                                                                         batch);
    count_launch();
    return cstat(cudaGetLastError());
}
