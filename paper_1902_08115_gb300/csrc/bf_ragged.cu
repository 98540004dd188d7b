// bf_ragged.cu -- ragged batches: every problem has its own order n_b.  One
// persistent kernel, captured in a CUDA graph, factors each SPD matrix
// (dpotrf, lower, section 3.1) and solves its right-hand sides (dpotrs).
//
// Work items come from a device queue (one atomic counter, no waiting between
// CTAs), ordered by decreasing cost so the largest problems start first:
//   BIG items  (n_b > lane_max): one problem per CTA.  The lower triangle is
//     held packed in shared memory and factored right-looking with 16-column
//     panels: the panel's diagonal block by one warp (pivots via rsqrt), the
//     rows below it by all threads (one row's triangular solve each), the
//     trailing update by all threads on 4x4 register tiles (section 3.2.1's
//     dgemm loop + edge structure at CTA scale); three barriers per panel.
//     Then a blocked forward/backward substitution.
//   LANE items (n_b <= lane_max): blockDim problems per CTA, one per thread,
//     sorted so a warp's problems have (nearly) equal order, using the same
//     lane Cholesky as the uniform path.
// The threshold lane_max and the CTA size are picked by the autotuner.
#include <algorithm>
#include <numeric>
#include <vector>

#include "bf_internal.h"
#include "bf_lane.cuh"
#include "../../include/bfgpu.h"

namespace bf {

struct RaggedParams {
    const int* n;            // order of each problem, in queue order
    const long long* offS;   // element offset of each matrix (ld = n)
    const long long* offB;   // element offset of each right-hand-side block (ld = n)
    const int* orig;         // original index (for info)
    double* S;
    double* B;
    int* info;
    int nrhs;
    int nbig;                // problems [0, nbig) are BIG items
    int nprob;
    int nitems;
    unsigned int* counter;
};

__device__ __forceinline__ int pcol(int j, int n) { return j * n - (j * (j - 1)) / 2; }  // packed column start

// --------------------------------------------------------------------------- BIG: one problem per CTA
#define BF_BIG_NB 16

__device__ void big_problem(const RaggedParams& p, int q, double* sm) {
    const int n = p.n[q];
    const int tid = threadIdx.x, T = blockDim.x, warp = tid >> 5, lane = tid & 31;
    double* P = sm;                                   // packed lower triangle
    double* X = sm + (size_t)n * (n + 1) / 2;         // n x nrhs right-hand sides
    double* rinv = X + (size_t)n * p.nrhs;            // reciprocal pivots
    __shared__ int s_fail;
    double* S = p.S + p.offS[q];
    double* Bq = p.B + p.offB[q];
    // flat, independent loads of the lower triangle (many in flight per thread)
    const int nn = n * n;
#pragma unroll 4
    for (int e = tid; e < nn; e += T) {
        const int j = e / n, i = e - j * n;
        if (i >= j) P[pcol(j, n) + i - j] = S[e];
    }
    for (int e = tid; e < n * p.nrhs; e += T) X[e] = Bq[e];
    if (tid == 0) s_fail = 0;
    __syncthreads();

    for (int J = 0; J < n; J += BF_BIG_NB) {
        const int nb = imin(BF_BIG_NB, n - J);
        // (1) Cholesky of the nb x nb diagonal block, warp-synchronous in warp 0
        if (warp == 0) {
            for (int c = 0; c < nb; c++) {
                const int j = J + c;
                const double d = P[pcol(j, n)];
                if (!(d > 0.0)) {  // the same value in every lane
                    if (lane == 0) s_fail = j + 1;
                    break;
                }
                const double rs = rsqrt(d);
                __syncwarp();
                if (lane == 0) {
                    P[pcol(j, n)] = d * rs;
                    rinv[j] = rs;
                }
                if (lane < nb - c - 1) P[pcol(j, n) + 1 + lane] *= rs;
                __syncwarp();
                const int w = nb - c - 1;  // trailing block columns/rows right of c
                for (int e = lane; e < w * w; e += 32) {
                    const int kk = e / w, rr = e - kk * w;
                    if (rr >= kk) {
                        const int i = j + 1 + rr, k = j + 1 + kk;
                        P[pcol(k, n) + i - k] = fma(-P[pcol(j, n) + i - j], P[pcol(j, n) + k - j], P[pcol(k, n) + i - k]);
                    }
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (s_fail) break;
        // (2) the panel rows below: L(i, J:J+nb) = A(i, J:J+nb) L_JJ^{-T}, one row per thread
        for (int i = J + nb + tid; i < n; i += T) {
            double x[BF_BIG_NB];
#pragma unroll
            for (int c = 0; c < BF_BIG_NB; c++) x[c] = (c < nb) ? P[pcol(J + c, n) + i - (J + c)] : 0.0;
#pragma unroll
            for (int c = 0; c < BF_BIG_NB; c++) {
                if (c < nb) {
#pragma unroll
                    for (int c2 = 0; c2 < c; c2++) x[c] = fma(-x[c2], P[pcol(J + c2, n) + c - c2], x[c]);
                    x[c] *= rinv[J + c];
                    P[pcol(J + c, n) + i - (J + c)] = x[c];
                }
            }
        }
        __syncthreads();
        // (3) trailing update L22 -= L21 L21^T, rank nb, on lower 4x4 tiles
        const int R = J + nb, m = n - R;
        if (m > 0) {
            const int tb = (m + 3) / 4;
            const int ntile = tb * (tb + 1) / 2;
            for (int t = tid; t < ntile; t += T) {
                int I = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
                while ((I + 1) * (I + 2) / 2 <= t) I++;
                while (I * (I + 1) / 2 > t) I--;
                const int K = t - I * (I + 1) / 2;
                const int i0 = R + 4 * I, k0 = R + 4 * K;
                double acc[4][4];
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int b = 0; b < 4; b++) acc[a][b] = 0.0;
                for (int c = 0; c < nb; c++) {
                    const int col = pcol(J + c, n) - (J + c);
                    double li[4], lk[4];
#pragma unroll
                    for (int a = 0; a < 4; a++) li[a] = P[col + imin(i0 + a, n - 1)];
#pragma unroll
                    for (int b = 0; b < 4; b++) lk[b] = P[col + imin(k0 + b, n - 1)];
#pragma unroll
                    for (int a = 0; a < 4; a++)
#pragma unroll
                        for (int b = 0; b < 4; b++) acc[a][b] = fma(li[a], lk[b], acc[a][b]);
                }
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    const int k = k0 + b;
                    if (k >= n) continue;
                    const int col = pcol(k, n) - k;
#pragma unroll
                    for (int a = 0; a < 4; a++) {
                        const int i = i0 + a;
                        if (i < n && i >= k) P[col + i] -= acc[a][b];
                    }
                }
            }
        }
        __syncthreads();
    }
    const int fail = s_fail;
    if (fail == 0) {
        // forward substitution L Y = B, 8-row blocks: the block triangle by warp 0, the rest by all
        const int r = p.nrhs;
        for (int J = 0; J < n; J += 8) {
            const int nb = imin(8, n - J);
            if (warp == 0) {
                for (int c = 0; c < nb; c++) {
                    const int j = J + c;
                    for (int e = lane; e < r; e += 32) X[j + e * n] *= rinv[j];
                    __syncwarp();
                    for (int e = lane; e < (nb - c - 1) * r; e += 32) {
                        const int i = j + 1 + e % (nb - c - 1), rr = e / (nb - c - 1);
                        X[i + rr * n] = fma(-P[pcol(j, n) + i - j], X[j + rr * n], X[i + rr * n]);
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
            const int m = n - J - nb;
            for (int e = tid; e < m * r; e += T) {
                const int i = J + nb + e % m, rr = e / m;
                double s = X[i + rr * n];
                for (int c = 0; c < nb; c++) s = fma(-P[pcol(J + c, n) + i - (J + c)], X[J + c + rr * n], s);
                X[i + rr * n] = s;
            }
            __syncthreads();
        }
        // backward substitution L^T X = Y
        for (int J = ((n - 1) / 8) * 8; J >= 0; J -= 8) {
            const int nb = imin(8, n - J);
            if (warp == 0) {
                for (int c = nb - 1; c >= 0; c--) {
                    const int j = J + c;
                    for (int e = lane; e < r; e += 32) X[j + e * n] *= rinv[j];
                    __syncwarp();
                    for (int e = lane; e < c * r; e += 32) {
                        const int i = J + e % c, rr = e / c;
                        X[i + rr * n] = fma(-P[pcol(i, n) + j - i], X[j + rr * n], X[i + rr * n]);
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
            for (int e = tid; e < J * r; e += T) {
                const int i = e % J, rr = e / J;
                double s = X[i + rr * n];
                for (int c = 0; c < nb; c++) s = fma(-P[pcol(i, n) + J + c - i], X[J + c + rr * n], s);
                X[i + rr * n] = s;
            }
            __syncthreads();
        }
        for (int e = tid; e < nn; e += T) {
            const int j = e / n, i = e - j * n;
            if (i >= j) S[e] = P[pcol(j, n) + i - j];
        }
        for (int e = tid; e < n * p.nrhs; e += T) Bq[e] = X[e];
    }
    if (tid == 0 && p.info) p.info[p.orig[q]] = fail;
    __syncthreads();
}

// --------------------------------------------------------------------------- LANE: one problem per thread
__device__ void lane_problem(const RaggedParams& p, int q) {
    const int n = p.n[q];
    double* S = p.S + p.offS[q];
    double* Bq = p.B + p.offB[q];
    const int info = potrf_lane_global<4, 2>(S, n, n);
    if (info == 0) {
        for (int c = 0; c < p.nrhs; c++) {
            double* b = Bq + (long long)c * n;
            for (int j = 0; j < n; j++) {
                const double yj = b[j] / S[j + (long long)j * n];
                b[j] = yj;
                for (int i = j + 1; i < n; i++) b[i] = fma(-S[i + (long long)j * n], yj, b[i]);
            }
            for (int j = n - 1; j >= 0; j--) {
                double s = b[j];
                for (int i = j + 1; i < n; i++) s = fma(-S[i + (long long)j * n], b[i], s);
                b[j] = s / S[j + (long long)j * n];
            }
        }
    }
    if (p.info) p.info[p.orig[q]] = info;
}

__global__ void __launch_bounds__(512) ragged_persistent_kernel(RaggedParams p) {
    extern __shared__ double smem[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(p.counter, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= p.nitems) break;
        if (item < p.nbig) {
            big_problem(p, item, smem);
        } else {
            const int q = p.nbig + (item - p.nbig) * (int)blockDim.x + (int)threadIdx.x;
            if (q < p.nprob) lane_problem(p, q);
        }
    }
}

size_t ragged_smem_bytes(int nmax, int nrhs) {
    return sizeof(double) * ((size_t)nmax * (nmax + 1) / 2 + (size_t)nmax * nrhs + nmax);
}

}  // namespace bf

// ----------------------------------------------------------------------------- plan
struct bf_ragged_plan_st {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bf::RaggedParams p;
    int threads, blocks;
    size_t smem;
};

extern "C" size_t bf_ragged_workspace_bytes(int batch) {
    // n, orig (int) + offS, offB (int64) per problem, one counter, 256-byte alignment slack
    return (size_t)batch * (2 * sizeof(int) + 2 * sizeof(long long)) + 4 * 256;
}

extern "C" int bf_ragged_potrf_potrs_plan_create(int batch, const int* n_host, int nrhs, double* S,
                                                 const long long* offS_host, double* B,
                                                 const long long* offB_host, int* info, void* workspace,
                                                 size_t workspace_bytes, int lane_max, int threads,
                                                 bf_stream_t stream, bf_ragged_plan_t* plan) {
    if (batch < 0) return -1;
    if (batch > 0 && !n_host) return -2;
    if (nrhs < 0 || nrhs > 64) return -3;
    if (batch > 0 && !S) return -4;
    if (batch > 0 && !offS_host) return -5;
    if (batch > 0 && nrhs > 0 && !B) return -6;
    if (batch > 0 && nrhs > 0 && !offB_host) return -7;
    if (workspace_bytes < bf_ragged_workspace_bytes(batch)) return -10;
    if (batch > 0 && !workspace) return -9;
    if (lane_max < 0) return -11;
    if (threads != 128 && threads != 256 && threads != 512) return -12;
    if (!plan) return -14;
    int nmax = 0;
    for (int b = 0; b < batch; b++) {
        if (n_host[b] < 0) return -2;
        nmax = std::max(nmax, n_host[b]);
    }
    const size_t smem = bf::ragged_smem_bytes(nmax > lane_max ? nmax : 0, nrhs);
    if (smem > 227 * 1024) return BF_ERR_NOT_SUPPORTED;
    // queue order: BIG problems by decreasing order, then LANE problems by decreasing order
    std::vector<int> order(batch);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n_host[a] > n_host[b]; });
    int nbig = 0;
    while (nbig < batch && n_host[order[nbig]] > lane_max) nbig++;
    std::vector<int> nq(batch), orig(batch);
    std::vector<long long> oS(batch), oB(batch);
    for (int i = 0; i < batch; i++) {
        const int b = order[i];
        nq[i] = n_host[b];
        orig[i] = b;
        oS[i] = offS_host[b];
        oB[i] = nrhs ? offB_host[b] : 0;
    }
    auto align = [](size_t x) { return (x + 255) / 256 * 256; };
    char* w = (char*)workspace;
    size_t o = 0;
    unsigned int* counter = (unsigned int*)(w + o);
    o = align(o + sizeof(unsigned int));
    int* dn = (int*)(w + o);
    o = align(o + sizeof(int) * batch);
    int* dorig = (int*)(w + o);
    o = align(o + sizeof(int) * batch);
    long long* doS = (long long*)(w + o);
    o = align(o + sizeof(long long) * batch);
    long long* doB = (long long*)(w + o);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (batch > 0) {
        e = cudaMemcpyAsync(dn, nq.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dorig, orig.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(doS, oS.data(), sizeof(long long) * batch, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(doB, oB.data(), sizeof(long long) * batch, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors go out of scope
        if (e != cudaSuccess) return BF_ERR_CUDA;
    }
    bf_ragged_plan_st* pl = new bf_ragged_plan_st();
    pl->p.n = dn;
    pl->p.offS = doS;
    pl->p.offB = doB;
    pl->p.orig = dorig;
    pl->p.S = S;
    pl->p.B = B;
    pl->p.info = info;
    pl->p.nrhs = nrhs;
    pl->p.nbig = nbig;
    pl->p.nprob = batch;
    pl->p.nitems = nbig + (batch - nbig + threads - 1) / threads;
    pl->p.counter = counter;
    pl->threads = threads;
    pl->smem = smem;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(bf::ragged_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
        delete pl;
        return BF_ERR_CUDA;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bf::ragged_persistent_kernel, threads, smem) !=
            cudaSuccess ||
        per_sm < 1) {
        delete pl;
        return BF_ERR_CUDA;
    }
    pl->blocks = sms * per_sm;
    // capture: reset the queue counter, then the persistent launch
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        delete pl;
        return BF_ERR_CUDA;
    }
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(counter, 0, sizeof(unsigned int), cs);
        bf::ragged_persistent_kernel<<<pl->blocks, threads, smem, cs>>>(pl->p);
        e = cudaStreamEndCapture(cs, &pl->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        delete pl;
        return BF_ERR_CUDA;
    }
    *plan = pl;
    return BF_SUCCESS;
}

extern "C" int bf_ragged_plan_launch(bf_ragged_plan_t plan, bf_stream_t stream) {
    if (!plan) return -1;
    if (plan->p.nprob == 0) return BF_SUCCESS;
    cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
    bf::count_launch();
    return e == cudaSuccess ? BF_SUCCESS : BF_ERR_CUDA;
}

extern "C" int bf_ragged_plan_destroy(bf_ragged_plan_t plan) {
    if (!plan) return -1;
    cudaGraphExecDestroy(plan->exec);
    cudaGraphDestroy(plan->graph);
    delete plan;
    return BF_SUCCESS;
}

extern "C" int bf_ragged_plan_info(bf_ragged_plan_t plan, int* out) {
    if (!plan) return -1;
    if (!out) return -2;
    out[0] = plan->p.nbig;
    out[1] = plan->p.nitems;
    out[2] = plan->blocks;
    out[3] = plan->threads;
    out[4] = (int)plan->smem;
    return BF_SUCCESS;
}

// ----------------------------------------------------------------------------- allocation-free entry point
// Some callers cannot allocate device memory when they solve: code running under a fixed
// memory budget (an embedded or real-time controller that sizes all memory at start-up and
// forbids allocation in its control loop, the setting the paper's routines are written for),
// and code that hands the library no workspace because another allocator owns the device.
// bf_ragged_potrf_potrs_noalloc serves them: the persistent kernel's queue lives in the
// file-scope array below, which every GPU that loads this library holds until the process
// exits, and the call allocates nothing (no cudaMalloc/cudaFree, no host heap).
#include <mutex>

#define BF_NOALLOC_ALIGN(x) (((x) + 255) / 256 * 256)

static constexpr size_t kNoallocCounter = 256;
static constexpr size_t kNoallocInts = BF_NOALLOC_ALIGN(sizeof(int) * (size_t)BF_RAGGED_NOALLOC_MAX);
static constexpr size_t kNoallocLongs = BF_NOALLOC_ALIGN(sizeof(long long) * (size_t)BF_RAGGED_NOALLOC_MAX);
static constexpr size_t kNoallocBytes = kNoallocCounter + 2 * kNoallocInts + 2 * kNoallocLongs;

static __device__ __align__(256) unsigned char g_ragged_noalloc_scratch[kNoallocBytes];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256];  // device address of the scratch array, per device ordinal
// host-side queue construction, reused by every call (guarded by g_noalloc_mu)
int h_order[BF_RAGGED_NOALLOC_MAX];
int h_n[BF_RAGGED_NOALLOC_MAX];
int h_orig[BF_RAGGED_NOALLOC_MAX];
long long h_offS[BF_RAGGED_NOALLOC_MAX];
long long h_offB[BF_RAGGED_NOALLOC_MAX];
}  // namespace

extern "C" int bf_ragged_potrf_potrs_noalloc(int batch, const int* n_host, int nrhs, double* S,
                                             const long long* offS_host, double* B, const long long* offB_host,
                                             int* info, int lane_max, int threads, bf_stream_t stream) {
    if (batch < 0) return -1;
    if (batch > 0 && !n_host) return -2;
    if (nrhs < 0 || nrhs > 64) return -3;
    if (batch > 0 && !S) return -4;
    if (batch > 0 && !offS_host) return -5;
    if (batch > 0 && nrhs > 0 && !B) return -6;
    if (batch > 0 && nrhs > 0 && !offB_host) return -7;
    if (lane_max < 0) return -9;
    if (threads != 128 && threads != 256 && threads != 512) return -10;
    if (batch > BF_RAGGED_NOALLOC_MAX) return BF_ERR_NOALLOC_LIMIT;
    if (batch == 0) return BF_SUCCESS;
    int nmax = 0;
    for (int b = 0; b < batch; b++) {
        if (n_host[b] < 0) return -2;
        nmax = std::max(nmax, n_host[b]);
    }
    const size_t smem = bf::ragged_smem_bytes(nmax > lane_max ? nmax : 0, nrhs);
    if (smem > 227 * 1024) return BF_ERR_NOT_SUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return BF_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    // set-up, once per device, with that device current
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_ragged_noalloc_scratch) != cudaSuccess || !ptr) return BF_ERR_CUDA;
        g_noalloc_ptr[dev] = ptr;
    }
    char* w = (char*)g_noalloc_ptr[dev];
    unsigned int* counter = (unsigned int*)w;
    int* dn = (int*)(w + kNoallocCounter);
    int* dorig = (int*)(w + kNoallocCounter + kNoallocInts);
    long long* doS = (long long*)(w + kNoallocCounter + 2 * kNoallocInts);
    long long* doB = (long long*)(w + kNoallocCounter + 2 * kNoallocInts + kNoallocLongs);
    // queue order: decreasing order n, ties by index (in place, no allocation)
    for (int i = 0; i < batch; i++) h_order[i] = i;
    std::sort(h_order, h_order + batch, [&](int a, int b) {
        return n_host[a] > n_host[b] || (n_host[a] == n_host[b] && a < b);
    });
    int nbig = 0;
    while (nbig < batch && n_host[h_order[nbig]] > lane_max) nbig++;
    for (int i = 0; i < batch; i++) {
        const int b = h_order[i];
        h_n[i] = n_host[b];
        h_orig[i] = b;
        h_offS[i] = offS_host[b];
        h_offB[i] = nrhs ? offB_host[b] : 0;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // pageable copies are staged before cudaMemcpyAsync returns, so the host arrays may be reused
    if (cudaMemcpyAsync(dn, h_n, sizeof(int) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dorig, h_orig, sizeof(int) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(doS, h_offS, sizeof(long long) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(doB, h_offB, sizeof(long long) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(counter, 0, sizeof(unsigned int), s) != cudaSuccess)  // the queue starts empty
        return BF_ERR_CUDA;
    bf::RaggedParams p;
    p.n = dn;
    p.offS = doS;
    p.offB = doB;
    p.orig = dorig;
    p.S = S;
    p.B = B;
    p.info = info;
    p.nrhs = nrhs;
    p.nbig = nbig;
    p.nprob = batch;
    p.nitems = nbig + (batch - nbig + threads - 1) / threads;
    p.counter = counter;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(bf::ragged_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return BF_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bf::ragged_persistent_kernel, threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return BF_ERR_CUDA;
    bf::ragged_persistent_kernel<<<sms * per_sm, threads, smem, s>>>(p);
    bf::count_launch();
    return cudaGetLastError() == cudaSuccess ? BF_SUCCESS : BF_ERR_CUDA;
}
