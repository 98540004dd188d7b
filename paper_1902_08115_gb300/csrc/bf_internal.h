// bf_internal.h -- declarations shared by the CUDA translation units of the
// library (not part of the public C ABI, which is include/bfgpu.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "bf_common.cuh"

namespace bf {

// Kernel variants the size switch chooses between (section 2.4: direct 'D'
// for very small sizes, packing variants for larger ones).
enum Variant : int { VAR_DIRECT = 0, VAR_PACKED = 1, VAR_BLOCKED = 2, VAR_TINY = 3, VAR_CTA = 4, VAR_TEAM = 5,
                     VAR_GROUP = 6 };

struct GemmConfig {
    int variant;  // VAR_DIRECT or VAR_PACKED
    int TM, TN;   // super-tile of C covered by one CTA (multiples of 4)
    int KC;       // k-slice staged in shared memory (packed)
    int P;        // problems per CTA
};

struct GemmParams {
    int m, n, k;
    double alpha, beta;
    int mode;
    MatRef A;
    int lda;
    MatRef B;
    int ldb;
    MatRef C;
    int ldc;
    long long batch;
    int TM, TN, KC, P;
    int tilesM, tilesN;
    int lower;
    const int* skip;
};

struct TrsmConfig {
    int variant;  // VAR_DIRECT or VAR_PACKED
    int MR;       // rows of the right-hand side per thread (4 or 8)
    int P;        // problems per CTA (packed)
    int minb;     // direct: 256-thread CTAs the kernel is compiled to keep per SM (1 or 2)
};

// Row-parallel triangular solve X T = alpha R (every row of R independent).
// T(p, j) = et ? A[j + p*lda] : A[p + j*lda]; R(r, j) = bt ? B[j + r*ldb] : B[r + j*ldb].
struct TrsmParams {
    int m, n;
    double alpha;
    MatRef A;
    int lda;
    MatRef B;
    int ldb;
    long long batch;
    int et, upper, unit, bt;
    int tpp;  // threads per problem = ceil(m / MR)
    int P;
    const int* skip;
    MatRef Bsrc;       // dtrmm only, when has_src: the input B (the result goes to B)
    int ldbs = 0;
    int has_src = 0;
};

struct PotrfConfig {
    int variant;  // VAR_DIRECT (lane per problem, in place), VAR_PACKED (lane per problem,
                  // shared memory), VAR_BLOCKED (right-looking sequence of kernels),
                  // VAR_CTA (problem per CTA, lower, n <= 256; small batches),
                  // VAR_TEAM (tpp lanes per problem; small batches of small orders)
    int T;        // threads (= problems) per CTA for the lane kernels
    int NB;       // block size of the blocked variant
    int rows;     // lane kernels: row-block height, 4 or 8
    int unroll;   // lane kernels: unroll of the k loops, 1 or 2
    int tpp = 4;  // VAR_TEAM: lanes per problem, 2 or 4
};

struct PotrfParams {
    int n;
    MatRef A;
    int lda;
    long long batch;
    int* info;      // per-problem LAPACK info (device), may be null
    int info_off;   // added to a failing column (blocked use on a sub-matrix)
    const int* skip;
    int upper;      // 1: A = U^T U from the upper triangle (the lower factor of the transposed view)
};

// SMs of a GB300.  Grid caps of grid-stride kernels and the batch-size switch points, all
// measured on this GPU, are expressed in it.  (The ragged plan queries the device instead,
// since its grid is exactly one wave of resident CTAs.)
constexpr long long kSMs = 152;

// Threads per CTA for a flat launch of `threads` independent threads.  With at least two
// CTAs of max_block per SM the launch keeps max_block.  Below that (a small batch, or a block
// of the blocked dtrsm) some SMs would idle, so the CTA size (max_block, 1/2, 1/4 or 1/8 of
// it) is the one that puts the fewest warps on the busiest of the 152 SMs, CTAs being dealt
// out evenly; a tie keeps the larger CTA.  E.g. 512 warps: 64 CTAs of 8 warps leave 88 SMs
// idle and 8 warps on the others, 128 CTAs of 4 warps put 4 on every SM (dtrsm, n = 48 x
// 1,365 problems: 484 -> 753 GFLOP/s on GB300).  Any smaller size that does not lower that
// count measured slower (9 warps on the busiest SM instead of 8: 780 -> 626).
inline int spread_block(long long threads, int max_block) {
    const long long sms = kSMs;
    const long long W = (threads + 31) / 32;
    const int wmax = max_block / 32;
    if ((W + wmax - 1) / wmax >= 2 * sms) return max_block;
    int best_w = wmax;
    long long best = -1;
    for (int w = wmax; w >= 1; w /= 2) {
        const long long ctas = (W + w - 1) / w;
        const long long load = w * ((ctas + sms - 1) / sms);  // warps on the busiest SM
        if (best < 0 || load < best) {
            best = load;
            best_w = w;
        }
    }
    return 32 * best_w;
}

// Kernels may declare static shared memory too (a few flags and scratch words, well under
// 1 KB); the opt-in for more than the default 48 KB of dynamic shared memory is taken whenever
// the dynamic part comes within this much of 48 KB, so that the sum never exceeds the default.
constexpr size_t kStaticSmemSlack = 1024;

// Increments the library's kernel-launch counter (bf_launch_count).
void count_launch();

size_t gemm_smem_bytes(const GemmConfig& c);

cudaError_t launch_dgemm(bool ta, bool tb, int m, int n, int k, double alpha, MatRef A, int lda,
                         MatRef B, int ldb, double beta, MatRef C, int ldc, long long batch,
                         const GemmConfig& cfg, int lower, const int* skip, cudaStream_t s);

// side: 0 = left, 1 = right; uplo: 0 = lower, 1 = upper; trans, unit: 0/1
cudaError_t launch_dtrsm(int side, int uplo, int trans, int unit, int m, int n, double alpha,
                         MatRef A, int lda, MatRef B, int ldb, long long batch,
                         const TrsmConfig& cfg, const int* skip, cudaStream_t s);

cudaError_t launch_dpotrf_lane(int n, MatRef A, int lda, long long batch, int* info, int info_off,
                               const int* skip, const PotrfConfig& cfg, cudaStream_t s, int upper = 0);

cudaError_t launch_dpotrf(int n, MatRef A, int lda, long long batch, int* info,
                          const PotrfConfig& cfg, cudaStream_t s, int upper = 0);

// tiny problems, one per thread through shared memory (bf_tiny.cu): dgemm with m, n, k <= 4,
// dtrsm with both orders <= 8
cudaError_t launch_dgemm_tiny(bool ta, bool tb, bool neg, const GemmParams& p, cudaStream_t s);
size_t tiny_gemm_smem(int m, int n, int k, int T);
cudaError_t launch_dtrsm_tiny(int side, int uplo, int trans, int unit, int m, int n, double alpha, MatRef A, int lda,
                              MatRef B, int ldb, long long batch, const int* skip, cudaStream_t s);

// dsyrk (upper: 0/1, trans: 0/1) and the fused chol(C + A A^T), lower (bf_dsyrk.cu)
cudaError_t launch_dsyrk(int upper, int trans, int n, int k, double alpha, MatRef A, int lda, double beta,
                         MatRef C, int ldc, long long batch, cudaStream_t s, const MatRef* Cin = nullptr,
                         int ldcin = 0);  // Cin: C's old values read from there (the uplo triangle)
// Cin (optional): the lower triangle of C is taken from Cin (ld ldcin) instead of C itself.
// merged (optional, with stage >= 0): the Riccati recursion's stage-tagged status -- an entry
// that is still 0 becomes 1000 stage + this factorisation's info; `info` is then scratch.
cudaError_t launch_dsyrk_dpotrf(int n, int k, MatRef A, int lda, MatRef C, int ldc, long long batch, int* info,
                                cudaStream_t s, const MatRef* Cin = nullptr, int ldcin = 0, int* merged = nullptr,
                                int stage = -1);
// info[q] = 1000 stage + stage_info[q] where info[q] is 0 and stage_info[q] is not (bf_riccati.cu)
cudaError_t launch_merge_stage_info(const int* stage_info, int* info, int stage, long long batch, cudaStream_t s);

// dtrmm, row-parallel like dtrsm (bf_dtrmm.cu); side: 0 = left, 1 = right
cudaError_t launch_dtrmm(int side, int uplo, int trans, int unit, int m, int n, double alpha, MatRef A, int lda,
                         MatRef B, int ldb, long long batch, int MR, cudaStream_t s,
                         const MatRef* Bsrc = nullptr, int ldbs = 0);

// LU with partial pivoting and its solve (bf_dgetrf.cu); ipiv: sipiv ints per problem, 1-based
// m x n; m != n always takes one problem per CTA (m <= kGetrfMaxRows)
constexpr int kGetrfMaxRows = 1024;
// square orders up to this take the four-lanes-per-problem form in shared memory (VAR_TEAM)
constexpr int kGetrfTeamMaxN = 16;
cudaError_t launch_dgetrf(int m, int n, MatRef A, int lda, int* ipiv, long long sipiv, int* info, long long batch,
                          cudaStream_t s);
cudaError_t launch_dgetrs(int trans, int n, int nrhs, MatRef A, int lda, const int* ipiv, long long sipiv, MatRef B,
                          int ldb, long long batch, cudaStream_t s);

// Configuration choice (the size switch), in bf_tune.cu.
GemmConfig choose_gemm(bool ta, bool tb, int m, int n, int k, int lda, long long batch);
TrsmConfig choose_trsm(int side, int uplo, int trans, int unit, int m, int n, long long batch);
// allow_group = false: the choice among the other forms (for sub-problems such as the blocked
// form's diagonal blocks, which are factored in place inside a larger matrix)
PotrfConfig choose_potrf(int n, int lda, long long batch, bool allow_group = true);
int choose_getrf(int n, long long batch);  // VAR_DIRECT (lane LU), VAR_TEAM (n <= 16) or VAR_CTA
// dpotrf of a group of problems per CTA in shared memory, element-parallel (bf_potrf_group.cu);
// kGroupSmemMax bounds its shared memory (one group must fit: potrf_group_smem(n, 1))
constexpr size_t kGroupSmemMax = 227 * 1024;
size_t potrf_group_smem(int n, int P);
int potrf_group_size(int n, long long batch, int per_sm);
cudaError_t launch_dpotrf_group(int n, MatRef A, int lda, long long batch, int* info, cudaStream_t s, int upper,
                                int threads, int per_sm);
// dpotrf with one problem per CTA, n <= 256 (bf_ragged.cu); upper: A = U^T U from the upper
// triangle (the lower factorisation of the transposed view)
cudaError_t launch_dpotrf_cta(int n, MatRef A, int lda, long long batch, int* info, cudaStream_t s, int upper);
// dpotrf of a variable-size batch (device arrays n, Aarray, lda; max_n <= BF_VBATCHED_POTRF_NMAX)
cudaError_t launch_dpotrf_vbatched(const int* n, double* const* A, const int* lda, int* info, long long batch,
                                   int max_n, cudaStream_t s, int upper);

}  // namespace bf
