// bf_dpotrf.cu -- batched FP64 Cholesky, lower (section 3.1 "dpotrf").
//
// The paper implements dpotrf as nested loops of tailored kernels whose block
// size is the kernel size, each kernel being "dgemm_nt inner loop, then a
// register-resident edge, then a (lower) store" (section 3.2.1, the
// kernel_dpotrf_nt_l listing).  Here:
//
//  * lane kernels (small n): one thread factors one whole problem, so all 32
//    lanes of a warp execute the same FP64 instruction stream on 32 problems
//    (on this GPU an FP64 warp instruction costs the same whatever its active
//    mask, so per-problem lanes are the only way to keep the triangular loop
//    and the pivot square roots fully utilised).  Left-looking by 4-column
//    blocks: for the diagonal block, D = A_JJ - L_J L_J^T (dgemm loop), then
//    a 4x4 Cholesky in registers (edge); for each 4-row block below it,
//    acc = A_IJ - L_I L_J^T (dgemm loop), then acc L_JJ^{-T} (trsm edge).
//    DIRECT works in place in global memory; PACKED first copies the CTA's
//    problems into shared memory, problem-interleaved so that the 32 lanes
//    of a warp touch 32 consecutive words.
//
//  * blocked (large n, small batches): right-looking with block NB, as a
//    sequence of launches of the library's own kernels on sub-matrices --
//    lane Cholesky of the NB x NB diagonal blocks, row-parallel trsm of the
//    panel below, dsyrk trailing update on the triangle's tiles.
//
// info follows LAPACK: 0, or the 1-based column j whose pivot is not
// positive (or NaN); the problem's factorisation stops there.
#include "bf_internal.h"
#include "bf_lane.cuh"
#include "bf_stage.cuh"

namespace bf {

template <int R, int U, bool UP>
__global__ void __launch_bounds__(256) dpotrf_lane_direct_kernel(PotrfParams p) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= p.batch) return;
    if (p.skip && p.skip[q] != 0) return;
    const int info = UP ? potrf_lane<R, U>(GAccT{p.A.mptr(q), p.lda}, p.n)
                        : potrf_lane_global<R, U>(p.A.mptr(q), p.lda, p.n);
    if (info && p.info) p.info[q] = info + p.info_off;
}

// TEAM: TPP consecutive lanes per problem (bf_lane.cuh, potrf_team).  A team never straddles
// two warps: the CTA is whole warps and TPP divides 32.
template <int TPP, bool UP>
__global__ void __launch_bounds__(256) dpotrf_team_kernel(PotrfParams p) {
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long q = gt / TPP;
    const int rr = (int)(gt % TPP);
    if (q >= p.batch) return;
    if (p.skip && p.skip[q] != 0) return;  // the whole team leaves
    const int lane = (int)(threadIdx.x & 31);
    const unsigned mask = ((1u << TPP) - 1u) << (lane & ~(TPP - 1));
    const int info = UP ? potrf_team<TPP, 2>(GAccT{p.A.mptr(q), p.lda}, p.n, rr, mask)
                        : potrf_team_global<TPP, 2>(p.A.mptr(q), p.lda, p.n, rr, mask);
    if (info && p.info && rr == 0) p.info[q] = info + p.info_off;
}

// PACKED: the CTA's problems staged through shared memory (bf_stage.cuh: coalesced 16-byte
// loads when they are one contiguous run, a padded problem-interleaved layout), factored
// there one per thread, and written back the same way.
__global__ void __launch_bounds__(256) dpotrf_lane_packed_kernel(PotrfParams p) {
    extern __shared__ double smem[];
    const int T = blockDim.x, ST = T + 1;
    const long long q0 = blockIdx.x * (long long)T;
    const int n = p.n;
    const int nq = (int)((p.batch - q0) < T ? (p.batch - q0) : T);
    const bool up = p.upper != 0;
    stage_in(p.A, n, n, p.lda, up, q0, nq, smem, ST);
    stage_wait();
    __syncthreads();
    const long long q = q0 + threadIdx.x;
    if ((int)threadIdx.x < nq && !(p.skip && p.skip[q] != 0)) {
        const int info = potrf_lane<4, 2>(SAcc{smem + threadIdx.x, n, ST}, n);
        if (info && p.info) p.info[q] = info + p.info_off;
    }
    __syncthreads();
    // back: the stored triangle; a contiguous lower batch goes back whole, the other triangle
    // with the very values it was read with
    stage_out(p.A, n, n, p.lda, up, q0, nq, smem, ST, !up, [](int i, int j) { return i >= j; });
}

template <bool UP>
static void launch_direct(const PotrfParams& p, const PotrfConfig& cfg, unsigned blocks, int T, cudaStream_t s) {
    if (cfg.rows == 8) {
        if (cfg.unroll == 2) {
            dpotrf_lane_direct_kernel<8, 2, UP><<<blocks, T, 0, s>>>(p);
        } else {
            dpotrf_lane_direct_kernel<8, 1, UP><<<blocks, T, 0, s>>>(p);
        }
    } else {
        if (cfg.unroll == 1) {
            dpotrf_lane_direct_kernel<4, 1, UP><<<blocks, T, 0, s>>>(p);
        } else {
            dpotrf_lane_direct_kernel<4, 2, UP><<<blocks, T, 0, s>>>(p);
        }
    }
}

cudaError_t launch_dpotrf_lane(int n, MatRef A, int lda, long long batch, int* info, int info_off,
                               const int* skip, const PotrfConfig& cfg, cudaStream_t s, int upper) {
    PotrfParams p;
    p.n = n; p.A = A; p.lda = lda; p.batch = batch; p.info = info; p.info_off = info_off; p.skip = skip;
    p.upper = upper;
    if (cfg.variant == VAR_PACKED) {
        const int T = cfg.T < 256 ? cfg.T : 256;
        size_t smem = sizeof(double) * (size_t)(T + 1) * n * n;
        if (smem + kStaticSmemSlack > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(dpotrf_lane_packed_kernel,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        long long blocks = (batch + T - 1) / T;
        dpotrf_lane_packed_kernel<<<(unsigned)blocks, T, smem, s>>>(p);
        count_launch();
        return cudaGetLastError();
    }
    const int T = cfg.T > 0 ? (cfg.T < 256 ? cfg.T / 32 * 32 : 256) : 128;  // the lane kernels' launch bounds
    if (cfg.variant == VAR_TEAM) {
        const int tpp = cfg.tpp == 2 ? 2 : 4;
        const unsigned blocks = (unsigned)((batch * tpp + T - 1) / T);
        if (tpp == 2) {
            if (upper) dpotrf_team_kernel<2, true><<<blocks, T, 0, s>>>(p);
            else dpotrf_team_kernel<2, false><<<blocks, T, 0, s>>>(p);
        } else {
            if (upper) dpotrf_team_kernel<4, true><<<blocks, T, 0, s>>>(p);
            else dpotrf_team_kernel<4, false><<<blocks, T, 0, s>>>(p);
        }
        count_launch();
        return cudaGetLastError();
    }
    const unsigned blocks = (unsigned)((batch + T - 1) / T);
    if (upper) {
        launch_direct<true>(p, cfg, blocks, T, s);
    } else {
        launch_direct<false>(p, cfg, blocks, T, s);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_dpotrf(int n, MatRef A, int lda, long long batch, int* info,
                          const PotrfConfig& cfg, cudaStream_t s, int upper) {
    if (batch == 0) return cudaSuccess;
    if (cfg.variant == VAR_GROUP) {
        if (potrf_group_smem(n, 1) <= kGroupSmemMax)  // writes every info itself
            return launch_dpotrf_group(n, A, lda, batch, info, s, upper, cfg.T, cfg.NB);
        PotrfConfig b = cfg;  // one problem does not fit in shared memory
        b.variant = n > 64 ? VAR_BLOCKED : VAR_DIRECT;
        b.T = 64;
        b.NB = 32;
        return launch_dpotrf(n, A, lda, batch, info, b, s, upper);
    }
    if (info) {
        cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int) * (size_t)batch, s);
        if (e != cudaSuccess) return e;
    }
    if (n == 0) return cudaSuccess;
    if (cfg.variant == VAR_CTA && n <= 256) return launch_dpotrf_cta(n, A, lda, batch, info, s, upper);
    if (cfg.variant == VAR_CTA) {  // too large for one CTA: blocked, or the lane kernel
        PotrfConfig b = cfg;
        b.variant = n > 64 ? VAR_BLOCKED : VAR_DIRECT;
        return launch_dpotrf(n, A, lda, batch, info, b, s, upper);
    }
    if (cfg.variant != VAR_BLOCKED) return launch_dpotrf_lane(n, A, lda, batch, info, 0, nullptr, cfg, s, upper);
    // right-looking blocked factorisation built from the library's kernels
    const int NB = cfg.NB;
    PotrfConfig lane = choose_potrf(NB, lda, batch, false);  // the diagonal blocks: lane or team form
    if (lane.variant != VAR_TEAM) lane.variant = VAR_DIRECT;
    for (int J = 0; J < n; J += NB) {
        const int jb = (n - J < NB) ? (n - J) : NB;
        cudaError_t e = launch_dpotrf_lane(jb, mat_sub(A, J, J, lda), lda, batch, info, J, info, lane, s, upper);
        if (e != cudaSuccess) return e;
        const int rest = n - J - jb;
        if (rest <= 0) break;
        if (upper) {
            // panel: U(J:J+jb, J+jb:n) = U_JJ^{-T} A(J:J+jb, J+jb:n)
            TrsmConfig tc = choose_trsm(0, 1, 1, 0, jb, rest, batch);
            e = launch_dtrsm(0, 1, 1, 0, jb, rest, 1.0, mat_sub(A, J, J, lda), lda,
                             mat_sub(A, J, J + jb, lda), lda, batch, tc, info, s);
            if (e != cudaSuccess) return e;
            // trailing update (upper triangle only, tiles of the triangle alone): A22 -= U12^T U12
            e = launch_dsyrk(1, 1, rest, jb, -1.0, mat_sub(A, J, J + jb, lda), lda, 1.0,
                             mat_sub(A, J + jb, J + jb, lda), lda, batch, s);
            if (e != cudaSuccess) return e;
            continue;
        }
        // panel: L(J+jb:n, J:J+jb) = A(J+jb:n, J:J+jb) L_JJ^{-T}
        TrsmConfig tc = choose_trsm(1, 0, 1, 0, rest, jb, batch);
        e = launch_dtrsm(1, 0, 1, 0, rest, jb, 1.0, mat_sub(A, J, J, lda), lda,
                         mat_sub(A, J + jb, J, lda), lda, batch, tc, info, s);
        if (e != cudaSuccess) return e;
        // trailing update (lower triangle only, tiles of the triangle alone): A22 -= L21 L21^T;
        // a problem that failed keeps being updated, harmlessly: its info is already set and
        // its later columns are unspecified (LAPACK)
        e = launch_dsyrk(0, 0, rest, jb, -1.0, mat_sub(A, J + jb, J, lda), lda, 1.0,
                         mat_sub(A, J + jb, J + jb, lda), lda, batch, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace bf
