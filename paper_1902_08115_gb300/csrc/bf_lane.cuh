// bf_lane.cuh -- the lane Cholesky: one thread factors one whole problem.
//
// Left-looking by 4-column blocks, in the structure of the paper's
// kernel_dpotrf_nt_l (section 3.2.1): the rows J..n-1 of block column J are
// computed as "dgemm_nt loop over the factored columns, then an edge".  Two
// row-block heights R:
//
//  * R = 4: the 4x4 diagonal block (Cholesky edge in registers), then 4x4
//    blocks below it (triangular edge with the reciprocal pivots).  Each k
//    step of a block moves 8 words for 16 fused multiply-adds.
//  * R = 8: the first row block holds the diagonal block and the 4 rows under
//    it, like the paper's 8x4 dpotrf kernel; the rows below follow as 8x4
//    blocks and a 4x4 tail.  Each k step of an 8x4 block moves 12 words for
//    32 fused multiply-adds, at the price of more registers per thread.
//
// Shared by the uniform (bf_dpotrf.cu), ragged (bf_ragged.cu) and fused dsyrk + dpotrf
// (bf_dsyrk.cu) kernels.
//
// Operands are reached through an accessor whose strip<R> loads move R
// consecutive rows of one column (rows clamped to n - 1 at the end of the
// matrix).  The lanes of a warp hold different problems, so every access is
// uncoalesced and these kernels are bound by L1 request throughput; the
// global accessors differ in how many requests a strip takes.
#pragma once

#include "bf_common.cuh"

namespace bf {

// Global memory, one 8-byte access per element.
struct GAccS {
    double* a;
    int lda;
    __device__ __forceinline__ double ld(int i, int j) const { return a[i + (long long)j * lda]; }
    __device__ __forceinline__ void st(int i, int j, double v) const { a[i + (long long)j * lda] = v; }
    template <int R>
    __device__ __forceinline__ void strip(int i, int j, int n, double* o) const {
#pragma unroll
        for (int r = 0; r < R; r++) o[r] = ld(imin(i + r, n - 1), j);
    }
    template <int R>
    __device__ __forceinline__ void put(int i, int j, int cnt, const double* v) const {
#pragma unroll
        for (int r = 0; r < R; r++)
            if (r < cnt) st(i + r, j, v[r]);
    }
};

// Global memory, base 16-byte aligned and lda even: every strip that starts at
// an even row is 16-byte aligned and moves as R/2 16-byte accesses.
struct GAccV {
    double* a;
    int lda;
    __device__ __forceinline__ double ld(int i, int j) const { return a[i + (long long)j * lda]; }
    __device__ __forceinline__ void st(int i, int j, double v) const { a[i + (long long)j * lda] = v; }
    template <int R>
    __device__ __forceinline__ void strip(int i, int j, int n, double* o) const {
        if (i + R <= n) {
            const double2* p = reinterpret_cast<const double2*>(a + i + (long long)j * lda);
#pragma unroll
            for (int k = 0; k < R / 2; k++) {
                const double2 x = p[k];
                o[2 * k] = x.x;
                o[2 * k + 1] = x.y;
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; r++) o[r] = ld(imin(i + r, n - 1), j);
        }
    }
    template <int R>
    __device__ __forceinline__ void put(int i, int j, int cnt, const double* v) const {
        if (cnt == R) {
            double2* p = reinterpret_cast<double2*>(a + i + (long long)j * lda);
#pragma unroll
            for (int k = 0; k < R / 2; k++) p[k] = make_double2(v[2 * k], v[2 * k + 1]);
        } else {
#pragma unroll
            for (int r = 0; r < R; r++)
                if (r < cnt) st(i + r, j, v[r]);
        }
    }
};

// Global memory, any lda: a strip moves as 16-byte pieces from its first
// 16-byte boundary on -- R/2 accesses when it starts on a boundary, R/2 + 1
// (a single word at each end) when it starts 8 bytes past one.
struct GAccP {
    double* a;
    int lda;
    __device__ __forceinline__ double ld(int i, int j) const { return a[i + (long long)j * lda]; }
    __device__ __forceinline__ void st(int i, int j, double v) const { a[i + (long long)j * lda] = v; }
    template <int R>
    __device__ __forceinline__ void strip(int i, int j, int n, double* o) const {
        const double* p = a + i + (long long)j * lda;
        if (i + R <= n) {
            if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
#pragma unroll
                for (int k = 0; k < R / 2; k++) {
                    const double2 x = reinterpret_cast<const double2*>(p)[k];
                    o[2 * k] = x.x;
                    o[2 * k + 1] = x.y;
                }
            } else {
                o[0] = p[0];
#pragma unroll
                for (int k = 0; k < R / 2 - 1; k++) {
                    const double2 x = reinterpret_cast<const double2*>(p + 1)[k];
                    o[1 + 2 * k] = x.x;
                    o[2 + 2 * k] = x.y;
                }
                o[R - 1] = p[R - 1];
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; r++) o[r] = ld(imin(i + r, n - 1), j);
        }
    }
    template <int R>
    __device__ __forceinline__ void put(int i, int j, int cnt, const double* v) const {
        double* p = a + i + (long long)j * lda;
        if (cnt == R) {
            if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
#pragma unroll
                for (int k = 0; k < R / 2; k++) reinterpret_cast<double2*>(p)[k] = make_double2(v[2 * k], v[2 * k + 1]);
            } else {
                p[0] = v[0];
#pragma unroll
                for (int k = 0; k < R / 2 - 1; k++)
                    reinterpret_cast<double2*>(p + 1)[k] = make_double2(v[1 + 2 * k], v[2 + 2 * k]);
                p[R - 1] = v[R - 1];
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; r++)
                if (r < cnt) p[r] = v[r];
        }
    }
};

struct SAcc {  // a problem in shared memory, interleaved with the CTA's other problems
    double* s;
    int n, T;
    __device__ __forceinline__ double ld(int i, int j) const { return s[(i + j * n) * T]; }
    __device__ __forceinline__ void st(int i, int j, double v) const { s[(i + j * n) * T] = v; }
    template <int R>
    __device__ __forceinline__ void strip(int i, int j, int nn, double* o) const {
#pragma unroll
        for (int r = 0; r < R; r++) o[r] = ld(imin(i + r, nn - 1), j);
    }
    template <int R>
    __device__ __forceinline__ void put(int i, int j, int cnt, const double* v) const {
#pragma unroll
        for (int r = 0; r < R; r++)
            if (r < cnt) st(i + r, j, v[r]);
    }
};

// Global memory, transposed view: element (i, j) of the view is a[j + i lda], so the lower
// Cholesky of the view reads and writes the upper triangle of the stored matrix (A = U^T U,
// U = the view's L transposed).  A strip runs along a row of the stored matrix: single words.
struct GAccT {
    double* a;
    int lda;
    // the k loops take columns in pairs: L(i, p) and L(i, p + 1) are adjacent in memory
    static constexpr bool kPairs = true;
    __device__ __forceinline__ double ld(int i, int j) const { return a[j + (long long)i * lda]; }
    __device__ __forceinline__ void st(int i, int j, double v) const { a[j + (long long)i * lda] = v; }
    template <int R>
    __device__ __forceinline__ void strip(int i, int j, int n, double* o) const {
#pragma unroll
        for (int r = 0; r < R; r++) o[r] = ld(imin(i + r, n - 1), j);
    }
    // the strips of columns p and p + 1 (p + 1 < n): one 16-byte load per row where aligned
    template <int R>
    __device__ __forceinline__ void strip2(int i, int p, int n, double* o0, double* o1) const {
#pragma unroll
        for (int r = 0; r < R; r++) {
            const double* q = a + p + (long long)imin(i + r, n - 1) * lda;
            if ((reinterpret_cast<uintptr_t>(q) & 15u) == 0) {
                const double2 x = *reinterpret_cast<const double2*>(q);
                o0[r] = x.x;
                o1[r] = x.y;
            } else {
                o0[r] = q[0];
                o1[r] = q[1];
            }
        }
    }
    template <int R>
    __device__ __forceinline__ void put(int i, int j, int cnt, const double* v) const {
#pragma unroll
        for (int r = 0; r < R; r++)
            if (r < cnt) st(i + r, j, v[r]);
    }
};

// Accessors that read a row's entries of two adjacent columns as one piece (kPairs, strip2):
// the k loops below then step two columns at a time, with the multiply-adds in the same order.
template <class A, class = void>
struct AccPairs {
    static constexpr bool value = false;
};
template <class A>
struct AccPairs<A, decltype(void(A::kPairs))> {
    static constexpr bool value = A::kPairs;
};

// The optional rank-k operand of the fused dsyrk + dpotrf: the factorisation then acts on
// C + Y Y^T, the product accumulated in the same register tiles as the Cholesky updates
// (the paper's fused dsyrk_dpotrf routine, section 5).  NoSyrk: plain dpotrf.
struct NoSyrk {
    static constexpr bool active = false;
    template <int R>
    __device__ __forceinline__ void strip(int, int, int, double* o) const {
#pragma unroll
        for (int r = 0; r < R; r++) o[r] = 0.0;
    }
};

template <class G>
struct SyrkOp {  // Y (n x k) in global memory through accessor G
    static constexpr bool active = true;
    G g;
    template <int R>
    __device__ __forceinline__ void strip(int i, int j, int n, double* o) const { g.template strip<R>(i, j, n, o); }
};

// acc (R x 4) <- acc L_JJ^{-T}: forward substitution against the factored
// diagonal block d (lower, diagonal replaced by its reciprocal rinv).
template <int R>
__device__ __forceinline__ void trsm_edge(double (&acc)[R][4], const double (&d)[4][4], const double (&rinv)[4]) {
#pragma unroll
    for (int c = 0; c < 4; c++) {
#pragma unroll
        for (int c2 = 0; c2 < c; c2++)
#pragma unroll
            for (int r = 0; r < R; r++) acc[r][c] = fma(-acc[r][c2], d[c][c2], acc[r][c]);
#pragma unroll
        for (int r = 0; r < R; r++) acc[r][c] *= rinv[c];
    }
}

// Rows I..I+R-1 of block column J: acc = A(I:I+R, J:J+4) - L(I:I+R, 0:J) L(J:J+4, 0:J)^T,
// then acc L_JJ^{-T}, stored for the rows that exist.  U = unroll of the k loop.
template <int R, int U, class Acc, class Y>
__device__ __forceinline__ void lane_block(const Acc& M, int n, int I, int J, int jb, const int (&jr)[4],
                                           const double (&d)[4][4], const double (&rinv)[4], const Y& ysk,
                                           int k) {
    double acc[R][4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        double col[R];
        M.template strip<R>(I, jr[c], n, col);
#pragma unroll
        for (int r = 0; r < R; r++) acc[r][c] = col[r];
    }
    if (Y::active) {
#pragma unroll U
        for (int p = 0; p < k; p++) {
            double a[R], b[4];
            ysk.template strip<R>(I, p, n, a);
            ysk.template strip<4>(J, p, n, b);
#pragma unroll
            for (int r = 0; r < R; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
    }
    // k in pairs through a pair accessor (J is a multiple of 4, so the pairs are whole)
    int pp0 = 0;
    if constexpr (AccPairs<Acc>::value) {
        for (; pp0 < J; pp0 += 2) {
            double a0[R], a1[R], b0[4], b1[4];
            M.template strip2<R>(I, pp0, n, a0, a1);
            M.template strip2<4>(J, pp0, n, b0, b1);
#pragma unroll
            for (int r = 0; r < R; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[r][c] = fma(-a0[r], b0[c], acc[r][c]);
#pragma unroll
            for (int r = 0; r < R; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[r][c] = fma(-a1[r], b1[c], acc[r][c]);
        }
    }
#pragma unroll U
    for (int pp = pp0; pp < J; pp++) {
        double a[R], b[4];
        M.template strip<R>(I, pp, n, a);
        M.template strip<4>(J, pp, n, b);
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[r][c] = fma(-a[r], b[c], acc[r][c]);
    }
    trsm_edge<R>(acc, d, rinv);
    const int ib = imin(R, n - I);
#pragma unroll
    for (int c = 0; c < 4; c++) {
        if (c < jb) {
            double col[R];
#pragma unroll
            for (int r = 0; r < R; r++) col[r] = acc[r][c];
            M.template put<R>(I, J + c, ib, col);
        }
    }
}

// D = A_JJ - L_J L_J^T (lower part) for the 4 rows J..J+3 alone.
template <int U, class Acc, class Y>
__device__ __forceinline__ void lane_diag(const Acc& M, int n, int J, const int (&jr)[4], double (&d)[4][4],
                                          const Y& ysk, int k) {
#pragma unroll
    for (int c = 0; c < 4; c++) {
        double col[4];
        M.template strip<4>(J, jr[c], n, col);  // rows above c are read but not used
#pragma unroll
        for (int r = c; r < 4; r++) d[r][c] = col[r];
    }
    if (Y::active) {
#pragma unroll U
        for (int p = 0; p < k; p++) {
            double l[4];
            ysk.template strip<4>(J, p, n, l);
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c <= r; c++) d[r][c] = fma(l[r], l[c], d[r][c]);
        }
    }
    int pp0 = 0;
    if constexpr (AccPairs<Acc>::value) {
        for (; pp0 < J; pp0 += 2) {
            double l0[4], l1[4];
            M.template strip2<4>(J, pp0, n, l0, l1);
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c <= r; c++) d[r][c] = fma(-l0[r], l0[c], d[r][c]);
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c <= r; c++) d[r][c] = fma(-l1[r], l1[c], d[r][c]);
        }
    }
#pragma unroll U
    for (int pp = pp0; pp < J; pp++) {
        double l[4];
        M.template strip<4>(J, pp, n, l);
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c <= r; c++) d[r][c] = fma(-l[r], l[c], d[r][c]);
    }
}

// Rows J..J+7 in one pass: D as above and E = A(J+4:J+8, J:J+4) - L(J+4:J+8, 0:J) L_J^T,
// both from one 8-row strip per k step.
template <int U, class Acc, class Y>
__device__ __forceinline__ void lane_diag_under(const Acc& M, int n, int J, const int (&jr)[4], double (&d)[4][4],
                                                double (&e)[4][4], const Y& ysk, int k) {
#pragma unroll
    for (int c = 0; c < 4; c++) {
        double col[8];
        M.template strip<8>(J, jr[c], n, col);  // rows above c are read but not used
#pragma unroll
        for (int r = c; r < 4; r++) d[r][c] = col[r];
#pragma unroll
        for (int r = 0; r < 4; r++) e[r][c] = col[4 + r];
    }
    if (Y::active) {
#pragma unroll U
        for (int p = 0; p < k; p++) {
            double l[8];
            ysk.template strip<8>(J, p, n, l);
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c <= r; c++) d[r][c] = fma(l[r], l[c], d[r][c]);
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) e[r][c] = fma(l[4 + r], l[c], e[r][c]);
        }
    }
    int pp0 = 0;
    if constexpr (AccPairs<Acc>::value) {
        for (; pp0 < J; pp0 += 2) {
            double l0[8], l1[8];
            M.template strip2<8>(J, pp0, n, l0, l1);
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const double* l = h ? l1 : l0;
#pragma unroll
                for (int r = 0; r < 4; r++)
#pragma unroll
                    for (int c = 0; c <= r; c++) d[r][c] = fma(-l[r], l[c], d[r][c]);
#pragma unroll
                for (int r = 0; r < 4; r++)
#pragma unroll
                    for (int c = 0; c < 4; c++) e[r][c] = fma(-l[4 + r], l[c], e[r][c]);
            }
        }
    }
#pragma unroll U
    for (int pp = pp0; pp < J; pp++) {
        double l[8];
        M.template strip<8>(J, pp, n, l);
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c <= r; c++) d[r][c] = fma(-l[r], l[c], d[r][c]);
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) e[r][c] = fma(-l[4 + r], l[c], e[r][c]);
    }
}

// 4x4 Cholesky edge in registers (rows past jb padded with the identity): d becomes L_JJ
// and rinv its reciprocal diagonal.  Returns 0, or the 1-based column (within the block)
// whose pivot is not positive.
__device__ __forceinline__ int chol_edge(double (&d)[4][4], double (&rinv)[4], int jb) {
#pragma unroll
    for (int r = 0; r < 4; r++) {
        if (r >= jb) {
#pragma unroll
            for (int c = 0; c < r; c++) d[r][c] = 0.0;
            d[r][r] = 1.0;
        }
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const double piv = d[c][c];
        if (!(piv > 0.0)) return c + 1;
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
    return 0;
}

// Factor one problem in place through the accessor, with row blocks of R (4 or 8) and the
// k loops unrolled U times.  Returns info (0 or 1-based column).
template <int R, int U, class Acc, class Y = NoSyrk>
__device__ __forceinline__ int potrf_lane(const Acc& M, int n, const Y& ysk = Y(), int k = 0) {
    for (int J = 0; J < n; J += 4) {
        const int jb = imin(4, n - J);
        const bool under = R == 8 && J + 4 < n;  // the 8-row first block applies
        int jr[4];
#pragma unroll
        for (int r = 0; r < 4; r++) jr[r] = imin(J + r, n - 1);
        double d[4][4], e[4][4], rinv[4];
        if (under) {
            lane_diag_under<U>(M, n, J, jr, d, e, ysk, k);
        } else {
            lane_diag<U>(M, n, J, jr, d, ysk, k);
        }
        const int f = chol_edge(d, rinv, jb);
        if (f) return J + f;
        // lower part of the diagonal block only (the strict upper triangle is never written)
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c <= r; c++)
                if (r < jb) M.st(J + r, J + c, d[r][c]);
        int I = J + 4;
        if (under) {  // the 4 rows under the diagonal block, accumulated with it
            trsm_edge<4>(e, d, rinv);
            const int ib = imin(4, n - I);
#pragma unroll
            for (int c = 0; c < 4; c++) {
                double col[4];
#pragma unroll
                for (int r = 0; r < 4; r++) col[r] = e[r][c];
                M.template put<4>(I, J + c, ib, col);
            }
            I += 4;
        }
        if (R == 8) {  // R-row blocks while more than 4 rows remain, then a 4-row tail
            for (; I + 4 < n; I += R) lane_block<R, U>(M, n, I, J, jb, jr, d, rinv, ysk, k);
        }
        for (; I < n; I += 4) lane_block<4, U>(M, n, I, J, jb, jr, d, rinv, ysk, k);
    }
    return 0;
}

// ---------------------------------------------------------------------------- team form
// TPP consecutive lanes of one warp (a team; TPP = 2 or 4) factor one problem together, for
// batches too small to give every FP64 pipe a warp of whole problems.  Per 4-column block J:
//  * D = A_JJ - L_J L_J^T: lane rr of the team takes the k = rr, rr + TPP, ... terms (lane 0
//    also the A_JJ term), and a butterfly of shuffles adds the partial sums.  Floating-point
//    addition is commutative, so every lane of the team ends with the same bits, takes the
//    same pivot decisions and leaves the loop at the same column;
//  * the 4-row blocks below are dealt round-robin to the team, each one the lane form's
//    dgemm loop and triangular edge;
//  * __syncwarp on the team's lanes orders the block column's stores before the next
//    block's loads (the team shares one SM, so one L1).
// Returns info (0 or the 1-based failing column), the same in every lane of the team.
template <int TPP, int U, class Acc>
__device__ __forceinline__ int potrf_team(const Acc& M, int n, int rr, unsigned mask) {
    for (int J = 0; J < n; J += 4) {
        const int jb = imin(4, n - J);
        int jr[4];
#pragma unroll
        for (int r = 0; r < 4; r++) jr[r] = imin(J + r, n - 1);
        double d[4][4], rinv[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            double col[4];
            M.template strip<4>(J, jr[c], n, col);  // rows above c are read but not used
#pragma unroll
            for (int r = c; r < 4; r++) d[r][c] = rr == 0 ? col[r] : 0.0;
        }
#pragma unroll U
        for (int pp = rr; pp < J; pp += TPP) {
            double l[4];
            M.template strip<4>(J, pp, n, l);
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c <= r; c++) d[r][c] = fma(-l[r], l[c], d[r][c]);
        }
#pragma unroll
        for (int o = 1; o < TPP; o <<= 1)
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c <= r; c++) d[r][c] += __shfl_xor_sync(mask, d[r][c], o);
        const int f = chol_edge(d, rinv, jb);
        if (f) return J + f;
        if (rr == 0) {
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c <= r; c++)
                    if (r < jb) M.st(J + r, J + c, d[r][c]);
        }
        for (int I = J + 4 + 4 * rr; I < n; I += 4 * TPP) lane_block<4, U>(M, n, I, J, jb, jr, d, rinv, NoSyrk(), 0);
        __syncwarp(mask);
    }
    return 0;
}

#ifndef BF_LANE8_MISALIGNED
#define BF_LANE8_MISALIGNED GAccP
#endif

// 16-byte alignment of every strip that starts at an even row: base aligned and lda even
__device__ __forceinline__ bool strips_aligned(const double* a, int lda) {
    return ((reinterpret_cast<unsigned long long>(a) & 15ull) == 0) && ((lda & 1) == 0);
}

// Factor one problem stored in global memory (any leading dimension).  Aligned problems
// take 16-byte strips; otherwise the 4-row form reads single words and the 8-row form
// 16-byte pieces from each strip's first boundary.
template <int R, int U>
__device__ __forceinline__ int potrf_lane_global(double* a, int lda, int n) {
    if (strips_aligned(a, lda)) return potrf_lane<R, U>(GAccV{a, lda}, n);
    if (R == 8) return potrf_lane<R, U>(BF_LANE8_MISALIGNED{a, lda}, n);
    return potrf_lane<R, U>(GAccS{a, lda}, n);
}

// The team form on a problem in global memory: 16-byte strips when aligned, else single words.
template <int TPP, int U>
__device__ __forceinline__ int potrf_team_global(double* a, int lda, int n, int rr, unsigned mask) {
    if (strips_aligned(a, lda)) return potrf_team<TPP, U>(GAccV{a, lda}, n, rr, mask);
    return potrf_team<TPP, U>(GAccS{a, lda}, n, rr, mask);
}

}  // namespace bf
