// bf_riccati.cu -- batched square-root Riccati recursion (section 5, "Riccati recursion"),
// the paper's application workload, as a sequence of the library's batched routines.
//
// Per problem: N stages, n_x states, n_u controls, m = n_u + n_x.  With Lc_N = chol(Q_N),
// for s = N-1 down to 0:
//   C   = [B_s^T; A_s^T] Lc_{s+1}          (dtrmm_rlnn, m x n_x)
//   F_s = chol([R_s S_s; S_s^T Q_s] + C C^T) (dsyrk_ln + dpotrf_l, fused or not)
//   Lc_s = the trailing n_x x n_x block of F_s
// Every launch covers the whole batch, so stage s of all problems runs at once; the
// stages themselves are sequential (each needs the previous factor).  A stage is two or three
// launches: the dtrmm reads [B^T; A^T]_s where it lies and writes C to the workspace, the
// factorisation reads the lower triangle of [R S; S^T Q]_s where it lies and writes F_s, and
// the fused kernel folds the stage-tagged status into info itself.  The fused form uses
// the fused dsyrk + dpotrf kernel (the paper's own-API routine, credited in section 5 with
// part of the speed-up over the plain BLAS/LAPACK calls); the unfused form calls dsyrk then
// dpotrf, as a BLAS/LAPACK implementation does.
#include "bf_internal.h"
#include "../../include/bfgpu.h"

namespace bf {

// dst(i, j) = src(i, j) for a rows x cols block of every problem
__global__ void copy_mat_kernel(int rows, int cols, const double* src, int lds, long long sS, double* dst, int ldd,
                                long long sD, long long batch) {
    const long long per = (long long)rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per * batch;
         e += (long long)gridDim.x * blockDim.x) {
        const long long q = e / per;
        const long long r = e - q * per;
        const int j = (int)(r / rows), i = (int)(r - (long long)j * rows);
        dst[q * sD + i + (long long)j * ldd] = src[q * sS + i + (long long)j * lds];
    }
}

// the first failing stage wins: info = 1000 stage + the stage's dpotrf info
__global__ void merge_info_kernel(const int* stage_info, int* info, int stage, long long batch) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q < batch && info[q] == 0 && stage_info[q] != 0) info[q] = 1000 * stage + stage_info[q];
}

static cudaError_t copy_mat(int rows, int cols, const double* src, int lds, long long sS, double* dst, int ldd,
                            long long sD, long long batch, cudaStream_t s) {
    const long long total = (long long)rows * cols * batch;
    if (total == 0) return cudaSuccess;
    int blocks = (int)((total + 255) / 256);
    if (blocks > kSMs * 32) blocks = kSMs * 32;
    copy_mat_kernel<<<blocks, 256, 0, s>>>(rows, cols, src, lds, sS, dst, ldd, sD, batch);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_merge_stage_info(const int* stage_info, int* info, int stage, long long batch, cudaStream_t s) {
    merge_info_kernel<<<(unsigned)((batch + 255) / 256), 256, 0, s>>>(stage_info, info, stage, batch);
    count_launch();
    return cudaGetLastError();
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace bf

using namespace bf;

extern "C" size_t bf_riccati_workspace_bytes(int nx, int nu, int batch) {
    if (nx < 0 || nu < 0 || batch < 0) return 0;
    const size_t m = (size_t)nx + nu;
    return align256(sizeof(double) * m * nx * batch) + align256(sizeof(int) * (size_t)batch);
}

extern "C" int bf_riccati_strided_batched(int N, int nx, int nu, const double* BAt, long long strideBAt,
                                          const double* RSQ, long long strideRSQ, const double* QN,
                                          long long strideQN, double* F, long long strideF, int* info, int fused,
                                          void* work, size_t work_bytes, int batch, bf_stream_t stream) {
    if (N < 0) return -1;
    if (nx < 1) return -2;
    if (nu < 0) return -3;
    const long long m = (long long)nx + nu;
    if (batch < 0) return -15;
    if (batch > 1 && strideBAt < (long long)N * m * nx) return -5;
    if (batch > 1 && strideRSQ < (long long)N * m * m) return -7;
    if (batch > 1 && strideQN < (long long)nx * nx) return -9;
    if (batch > 1 && strideF < (long long)(N + 1) * m * m) return -11;
    if (fused != 0 && fused != 1) return -13;
    if (batch == 0) return BF_SUCCESS;
    if ((N > 0 && (!BAt || !RSQ)) || !QN || !F) return N > 0 && !BAt ? -4 : (N > 0 && !RSQ ? -6 : (!QN ? -8 : -10));
    if (!info) return -12;
    if (work_bytes < bf_riccati_workspace_bytes(nx, nu, batch)) return -14;
    if (!work) return -14;
    cudaStream_t s = (cudaStream_t)stream;
    double* Cw = (double*)work;
    int* sinfo = (int*)((char*)work + align256(sizeof(double) * (size_t)m * nx * batch));
    const int mi = (int)m;
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    // terminal stage: F_N = [chol(Q_N) 0; 0 0]
    double* FN = F + (long long)N * m * m;
    if (!ok(cudaMemset2DAsync(FN, (size_t)strideF * sizeof(double), 0, (size_t)(m * m) * sizeof(double),
                              (size_t)batch, s)))
        return BF_ERR_CUDA;
    if (!ok(copy_mat(nx, nx, QN, nx, strideQN, FN, mi, strideF, batch, s))) return BF_ERR_CUDA;
    if (!ok(cudaMemsetAsync(info, 0, sizeof(int) * (size_t)batch, s))) return BF_ERR_CUDA;
    if (!ok(launch_dpotrf(nx, mat_strided(FN, strideF), mi, batch, sinfo, choose_potrf(nx, mi, batch), s)))
        return BF_ERR_CUDA;
    if (!ok(launch_merge_stage_info(sinfo, info, N, batch, s))) return BF_ERR_CUDA;
    for (int st = N - 1; st >= 0; st--) {
        double* Fs = F + (long long)st * m * m;
        const double* Lnext = (st + 1 == N) ? FN : F + (long long)(st + 1) * m * m + nu + (long long)nu * m;
        // C = BAt_s Lc_{s+1}: dtrmm out of place, BAt read where it is
        const MatRef bat = mat_strided(BAt + (long long)st * m * nx, strideBAt);
        if (!ok(launch_dtrmm(1, 0, 0, 0, mi, nx, 1.0, mat_strided(Lnext, strideF), mi, mat_strided(Cw, m * nx), mi,
                             batch, 4, s, &bat, mi)))
            return BF_ERR_CUDA;
        // F_s = chol(RSQ_s + C C^T): the lower triangle of RSQ_s read where it is
        const MatRef rsq = mat_strided(RSQ + (long long)st * m * m, strideRSQ);
        if (fused) {
            if (!ok(launch_dsyrk_dpotrf(mi, nx, mat_strided(Cw, m * nx), mi, mat_strided(Fs, strideF), mi, batch,
                                        sinfo, s, &rsq, mi, info, st)))
                return BF_ERR_CUDA;
        } else {
            if (!ok(launch_dsyrk(0, 0, mi, nx, 1.0, mat_strided(Cw, m * nx), mi, 1.0, mat_strided(Fs, strideF), mi,
                                 batch, s, &rsq, mi)))
                return BF_ERR_CUDA;
            if (!ok(launch_dpotrf(mi, mat_strided(Fs, strideF), mi, batch, sinfo, choose_potrf(mi, mi, batch), s)))
                return BF_ERR_CUDA;
            if (!ok(launch_merge_stage_info(sinfo, info, st, batch, s))) return BF_ERR_CUDA;
        }
    }
    return BF_SUCCESS;
}
