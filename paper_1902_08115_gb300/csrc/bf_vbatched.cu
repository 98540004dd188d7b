// bf_vbatched.cu -- variable-size batches ("vbatched"): every problem of the batch has its own
// sizes, leading dimensions and device pointers, read from device arrays, because the paper's
// matrices have sizes known only at run time (section 1).  The uniform batches carry the
// paper's kernels; here the problems of one launch differ, so the kernels read each problem's
// sizes and map threads to (problem, piece of work) pairs:
//   dgemm  -- one thread per 4x4 tile of C (section 2.1's register tile), the tiles numbered
//             densely across a chunk of problems (chunk_scan); the k loop reads op(A) and
//             op(B) from global memory (L1) as in the direct variant ('D', section 2.2);
//   dtrsm  -- one thread per independent row (right side) or column (left side) of B, the
//             paper's observation that right-side solves are independent row systems
//             (section 3.1 "dtrsm"), solved in place by substitution;
//   dpotrf -- csrc/bf_ragged.cu: one problem per thread up to order 32, else one per CTA.
// Illegal arguments of one problem (a size below zero or above its max_*, a leading dimension
// too small, a null pointer where data is needed) skip that problem and set its dinfo entry to
// minus the argument's position in the call; the other problems proceed.
#include "bf_internal.h"
#include "../../include/bfgpu.h"

namespace bf {

// Problems go in chunks of BF_VB_CH per CTA.  The chunk's units of work (tiles of C) are
// numbered densely across its problems, so a warp holds units of consecutive problems instead
// of idling on the lanes a smaller problem leaves empty.  s_start is the exclusive prefix sum
// of the units per problem (entries past the chunk are zero; two 32-entry warp scans by
// warp 0).  Small chunks keep many CTAs in flight.
#define BF_VB_CHUNK 64  // s_start entries
#define BF_VB_CH 8      // problems per chunk (measured: 8 beats 16, 32, 64 at 10k-100k problems)

__device__ __forceinline__ void chunk_scan(int* s_start) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        int a = s_start[lane + 1], b = s_start[lane + 33];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ua = __shfl_up_sync(0xffffffffu, a, o), ub = __shfl_up_sync(0xffffffffu, b, o);
            if (lane >= o) {
                a += ua;
                b += ub;
            }
        }
        b += __shfl_sync(0xffffffffu, a, 31);
        s_start[lane + 1] = a;
        s_start[lane + 33] = b;
        if (lane == 0) s_start[0] = 0;
    }
}

// the chunk problem holding unit u: the largest i with s_start[i] <= u
__device__ __forceinline__ int chunk_find(const int* s_start, int u) {
    int lo = 0, hi = BF_VB_CHUNK;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_start[mid] <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

struct VGemmParams {
    const int *m, *n, *k;
    double alpha, beta;
    const double* const* A;
    const int* lda;
    const double* const* B;
    const int* ldb;
    double* const* C;
    const int* ldc;
    int* dinfo;
    long long batch;
    int max_m, max_n, max_k;
};

// 0, or minus the position of the problem's first illegal argument
__device__ __forceinline__ int vgemm_check(const VGemmParams& p, bool ta, bool tb, long long q, int m, int n, int k) {
    if (m < 0 || m > p.max_m) return -3;
    if (n < 0 || n > p.max_n) return -4;
    if (k < 0 || k > p.max_k) return -5;
    const int ra = ta ? k : m, rb = tb ? n : k;
    if (p.lda[q] < (ra > 1 ? ra : 1)) return -8;
    if (p.ldb[q] < (rb > 1 ? rb : 1)) return -10;
    if (p.ldc[q] < (m > 1 ? m : 1)) return -13;
    const bool reads_ab = m > 0 && n > 0 && k > 0 && p.alpha != 0.0;
    if (reads_ab && !p.A[q]) return -7;
    if (reads_ab && !p.B[q]) return -9;
    if (m > 0 && n > 0 && !p.C[q]) return -12;
    return 0;
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) dgemm_vbatched_kernel(VGemmParams p) {
    __shared__ int s_start[BF_VB_CHUNK + 1];
    const int T = blockDim.x, tid = threadIdx.x;
    for (long long q0 = (long long)blockIdx.x * BF_VB_CH; q0 < p.batch; q0 += (long long)gridDim.x * BF_VB_CH) {
        if (tid < BF_VB_CHUNK) {  // tiles of each problem (0 when skipped or past the chunk); its status
            const long long q = q0 + tid;
            int cnt = 0;
            if (tid < BF_VB_CH && q < p.batch) {
                const int m = p.m[q], n = p.n[q], k = p.k[q];
                const int bad = vgemm_check(p, TA, TB, q, m, n, k);
                if (p.dinfo) p.dinfo[q] = bad;
                if (!bad) cnt = ((m + 3) / 4) * ((n + 3) / 4);
            }
            s_start[tid + 1] = cnt;
        }
        __syncthreads();
        chunk_scan(s_start);
        __syncthreads();
        const int total = s_start[BF_VB_CHUNK];
        for (int u = tid; u < total; u += T) {
            const int c = chunk_find(s_start, u);
            const long long q = q0 + c;
            const int t = u - s_start[c];
            const int m = p.m[q], n = p.n[q], k = p.k[q];
            const int tm = (m + 3) / 4;
            const int i0 = 4 * (t % tm), j0 = 4 * (t / tm);
            const double* A = p.A[q];
            const double* B = p.B[q];
            double* C = p.C[q];
            const int lda = p.lda[q], ldb = p.ldb[q], ldc = p.ldc[q];
            int ri[4], cj[4];
#pragma unroll
            for (int a = 0; a < 4; a++) {
                ri[a] = imin(i0 + a, m - 1);
                cj[a] = imin(j0 + a, n - 1);
            }
            // alpha == 1 with beta 0 or 1: the accumulators start from zero or C and are stored
            // as they are (no FP64 operation on the epilogue)
            const bool plain = p.alpha == 1.0 && (p.beta == 0.0 || p.beta == 1.0);
            double acc[4][4];
#pragma unroll
            for (int b = 0; b < 4; b++)
#pragma unroll
                for (int a = 0; a < 4; a++)
                    acc[a][b] = (plain && p.beta == 1.0) ? C[ri[a] + (long long)cj[b] * ldc] : 0.0;
            if (p.alpha != 0.0) {  // alpha == 0: A and B are not read
#pragma unroll 2
                for (int pp = 0; pp < k; pp++) {
                    double x[4], y[4];
#pragma unroll
                    for (int a = 0; a < 4; a++) {
                        x[a] = TA ? ldg(A + pp + (long long)ri[a] * lda) : ldg(A + ri[a] + (long long)pp * lda);
                        y[a] = TB ? ldg(B + cj[a] + (long long)pp * ldb) : ldg(B + pp + (long long)cj[a] * ldb);
                    }
#pragma unroll
                    for (int a = 0; a < 4; a++)
#pragma unroll
                        for (int b = 0; b < 4; b++) acc[a][b] = fma(x[a], y[b], acc[a][b]);
                }
            }
#pragma unroll
            for (int b = 0; b < 4; b++) {
#pragma unroll
                for (int a = 0; a < 4; a++) {
                    const int i = i0 + a, j = j0 + b;
                    if (i < m && j < n) {
                        double* cp = C + i + (long long)j * ldc;
                        if (plain) {
                            *cp = acc[a][b];
                        } else {
                            const double v = p.alpha * acc[a][b];
                            *cp = (p.beta == 0.0) ? v : fma(p.beta, *cp, v);  // beta == 0: C not read
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------ dtrsm
struct VTrsmParams {
    int right, lowerT, transA, unit;  // lowerT: op(A) lower
    const int *m, *n;
    double alpha;
    const double* const* A;
    const int* lda;
    double* const* B;
    const int* ldb;
    int* dinfo;
    long long batch;
    int max_m, max_n;
    int vmax;  // vector slots per problem: max_m (right side) or max_n (left side)
};

__device__ __forceinline__ int vtrsm_check(const VTrsmParams& p, long long q, int m, int n) {
    if (m < 0 || m > p.max_m) return -5;
    if (n < 0 || n > p.max_n) return -6;
    const int ka = p.right ? n : m;
    if (p.lda[q] < (ka > 1 ? ka : 1)) return -9;
    if (p.ldb[q] < (m > 1 ? m : 1)) return -11;
    if (m > 0 && n > 0 && p.alpha != 0.0 && !p.A[q]) return -8;
    if (m > 0 && n > 0 && !p.B[q]) return -10;
    return 0;
}

// one thread per (problem, vector): the vector is row v of B (right side: x op(A) = alpha b)
// or column v (left side: op(A) x = alpha b); x overwrites b, read back as it is solved.
// op(A)(i, j) = A(j, i) when transposed; lower op(A) is solved forward on the left and
// backward on the right, upper the other way round.
// one thread per (problem, vector), max_m (right side) or max_n (left side) slots per problem:
// a warp holds vectors of one problem, so its loads of op(A) are broadcasts and its loop
// lengths agree (numbering the vectors densely across problems measured 15 % slower)
__global__ void __launch_bounds__(128) dtrsm_vbatched_kernel(VTrsmParams p) {
    const long long total = p.batch * (long long)p.vmax;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long q = g / p.vmax;
        const int v = (int)(g - q * p.vmax);
        const int m = p.m[q], n = p.n[q];
        const int bad = vtrsm_check(p, q, m, n);
        if (v == 0 && p.dinfo) p.dinfo[q] = bad;
        if (bad || m == 0 || n == 0) continue;
        if (v >= (p.right ? m : n)) continue;
        const int len = p.right ? n : m, lda = p.lda[q], ldb = p.ldb[q];
        double* B = p.B[q];
        // x_e = B(v, e) (right) or B(e, v) (left)
        const long long xs = p.right ? ldb : 1;
        double* x = p.right ? B + v : B + (long long)v * ldb;
        if (p.alpha == 0.0) {  // B = 0, A not read
            for (int e = 0; e < len; e++) x[e * xs] = 0.0;
            continue;
        }
        const double* A = p.A[q];
        auto T = [&](int i, int j) -> double {  // op(A)(i, j)
            return p.transA ? ldg(A + j + (long long)i * lda) : ldg(A + i + (long long)j * lda);
        };
        // forward when (left, lower op(A)) or (right, upper op(A))
        const bool fwd = p.right ? !p.lowerT : p.lowerT;
        for (int t = 0; t < len; t++) {
            const int e = fwd ? t : len - 1 - t;
            double s = p.alpha * x[e * xs];
            if (fwd) {
                for (int f = 0; f < e; f++) s = fma(-x[f * xs], p.right ? T(f, e) : T(e, f), s);
            } else {
                for (int f = e + 1; f < len; f++) s = fma(-x[f * xs], p.right ? T(f, e) : T(e, f), s);
            }
            x[e * xs] = p.unit ? s : s / T(e, e);
        }
    }
}

// ------------------------------------------------------------------------------------ dpotrs
// Solve A X = B with the Cholesky factor of A (section 3.1 "dpotrf" and "dtrsm"): 'L' L Y = B then
// L^T X = Y; 'U' U^T Y = B then U X = Y.  One thread per (problem, right-hand side), both
// substitutions in the one launch, x overwriting b column by column.
struct VPotrsParams {
    int upper;
    const int *n, *nrhs;
    const double* const* A;
    const int* lda;
    double* const* B;
    const int* ldb;
    int* dinfo;
    long long batch;
    int max_n, max_nrhs;
};

__device__ __forceinline__ int vpotrs_check(const VPotrsParams& p, long long q, int n, int r) {
    if (n < 0 || n > p.max_n) return -2;
    if (r < 0 || r > p.max_nrhs) return -3;
    if (p.lda[q] < (n > 1 ? n : 1)) return -5;
    if (p.ldb[q] < (n > 1 ? n : 1)) return -7;
    if (n > 0 && r > 0 && !p.A[q]) return -4;
    if (n > 0 && r > 0 && !p.B[q]) return -6;
    return 0;
}

__global__ void __launch_bounds__(128) dpotrs_vbatched_kernel(VPotrsParams p) {
    const int vmax = p.max_nrhs > 0 ? p.max_nrhs : 1;
    const long long total = p.batch * (long long)vmax;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long q = g / vmax;
        const int c = (int)(g - q * vmax);
        const int n = p.n[q], r = p.nrhs[q];
        const int bad = vpotrs_check(p, q, n, r);
        if (c == 0 && p.dinfo) p.dinfo[q] = bad;
        if (bad || c >= r || n == 0) continue;
        const int lda = p.lda[q];
        const double* A = p.A[q];
        double* x = p.B[q] + (long long)c * p.ldb[q];
        // F(i, j) = the lower factor's (i, j), i >= j: L(i, j), or U(j, i) for 'U'
        auto F = [&](int i, int j) -> double {
            return p.upper ? ldg(A + j + (long long)i * lda) : ldg(A + i + (long long)j * lda);
        };
        for (int j = 0; j < n; j++) {  // forward: F y = b
            double s = x[j];
            for (int f = 0; f < j; f++) s = fma(-F(j, f), x[f], s);
            x[j] = s / F(j, j);
        }
        for (int j = n - 1; j >= 0; j--) {  // backward: F^T x = y
            double s = x[j];
            for (int f = j + 1; f < n; f++) s = fma(-F(f, j), x[f], s);
            x[j] = s / F(j, j);
        }
    }
}

cudaError_t launch_dpotrs_vbatched(const VPotrsParams& p, cudaStream_t s) {
    if (p.batch == 0) return cudaSuccess;
    const long long total = p.batch * (long long)(p.max_nrhs > 0 ? p.max_nrhs : 1);
    const int T = spread_block(total, 128);
    long long blocks = (total + T - 1) / T;
    if (blocks > kSMs * 64) blocks = kSMs * 64;
    dpotrs_vbatched_kernel<<<(unsigned)blocks, T, 0, s>>>(p);
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ launchers
cudaError_t launch_dgemm_vbatched(bool ta, bool tb, const VGemmParams& p0, cudaStream_t s) {
    if (p0.batch == 0) return cudaSuccess;
    VGemmParams p = p0;
    const int T = 128;
    long long blocks = (p.batch + BF_VB_CH - 1) / BF_VB_CH;
    if (blocks > kSMs * 64) blocks = kSMs * 64;
    if (ta) {
        if (tb) dgemm_vbatched_kernel<true, true><<<(unsigned)blocks, T, 0, s>>>(p);
        else dgemm_vbatched_kernel<true, false><<<(unsigned)blocks, T, 0, s>>>(p);
    } else {
        if (tb) dgemm_vbatched_kernel<false, true><<<(unsigned)blocks, T, 0, s>>>(p);
        else dgemm_vbatched_kernel<false, false><<<(unsigned)blocks, T, 0, s>>>(p);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_dtrsm_vbatched(const VTrsmParams& p0, cudaStream_t s) {
    if (p0.batch == 0) return cudaSuccess;
    VTrsmParams p = p0;
    p.vmax = p.right ? p.max_m : p.max_n;
    if (p.vmax < 1) p.vmax = 1;
    const long long total = p.batch * (long long)p.vmax;
    const int T = spread_block(total, 128);
    long long blocks = (total + T - 1) / T;
    if (blocks > kSMs * 64) blocks = kSMs * 64;
    dtrsm_vbatched_kernel<<<(unsigned)blocks, T, 0, s>>>(p);
    count_launch();
    return cudaGetLastError();
}

}  // namespace bf

// ------------------------------------------------------------------------------------ C ABI
using namespace bf;

static bool vb_trans(char c, bool* t) {
    if (c == 'N' || c == 'n') { *t = false; return true; }
    if (c == 'T' || c == 't' || c == 'C' || c == 'c') { *t = true; return true; }
    return false;
}

static int vb_status(cudaError_t e) { return e == cudaSuccess ? BF_SUCCESS : BF_ERR_CUDA; }

extern "C" int bf_dgemm_vbatched(char transa, char transb, const int* m, const int* n, const int* k, double alpha,
                                 const double* const* Aarray, const int* lda, const double* const* Barray,
                                 const int* ldb, double beta, double* const* Carray, const int* ldc, int batch,
                                 int max_m, int max_n, int max_k, int* dinfo, bf_stream_t stream) {
    bool ta, tb;
    if (!vb_trans(transa, &ta)) return -1;
    if (!vb_trans(transb, &tb)) return -2;
    if (batch < 0) return -14;
    if (max_m < 0) return -15;
    if (max_n < 0) return -16;
    if (max_k < 0) return -17;
    if (batch == 0) return BF_SUCCESS;
    if (!m) return -3;
    if (!n) return -4;
    if (!k) return -5;
    if (!Aarray) return -7;
    if (!lda) return -8;
    if (!Barray) return -9;
    if (!ldb) return -10;
    if (!Carray) return -12;
    if (!ldc) return -13;
    VGemmParams p{};
    p.m = m; p.n = n; p.k = k; p.alpha = alpha; p.beta = beta;
    p.A = Aarray; p.lda = lda; p.B = Barray; p.ldb = ldb; p.C = Carray; p.ldc = ldc;
    p.dinfo = dinfo; p.batch = batch; p.max_m = max_m; p.max_n = max_n; p.max_k = max_k;
    return vb_status(launch_dgemm_vbatched(ta, tb, p, (cudaStream_t)stream));
}

extern "C" int bf_dtrsm_vbatched(char side, char uplo, char transa, char diag, const int* m, const int* n,
                                 double alpha, const double* const* Aarray, const int* lda, double* const* Barray,
                                 const int* ldb, int batch, int max_m, int max_n, int* dinfo, bf_stream_t stream) {
    const bool right = side == 'R' || side == 'r', left = side == 'L' || side == 'l';
    if (!right && !left) return -1;
    const bool lower = uplo == 'L' || uplo == 'l', upper = uplo == 'U' || uplo == 'u';
    if (!lower && !upper) return -2;
    bool tr;
    if (!vb_trans(transa, &tr)) return -3;
    const bool unit = diag == 'U' || diag == 'u', nonunit = diag == 'N' || diag == 'n';
    if (!unit && !nonunit) return -4;
    if (batch < 0) return -12;
    if (max_m < 0) return -13;
    if (max_n < 0) return -14;
    if (batch == 0) return BF_SUCCESS;
    if (!m) return -5;
    if (!n) return -6;
    if (!Aarray) return -8;
    if (!lda) return -9;
    if (!Barray) return -10;
    if (!ldb) return -11;
    VTrsmParams p{};
    p.right = right; p.lowerT = lower != tr; p.transA = tr; p.unit = unit;
    p.m = m; p.n = n; p.alpha = alpha; p.A = Aarray; p.lda = lda; p.B = Barray; p.ldb = ldb;
    p.dinfo = dinfo; p.batch = batch; p.max_m = max_m; p.max_n = max_n;
    return vb_status(launch_dtrsm_vbatched(p, (cudaStream_t)stream));
}

extern "C" int bf_dpotrf_vbatched(char uplo, const int* n, double* const* Aarray, const int* lda, int* info,
                                  int batch, int max_n, bf_stream_t stream) {
    const bool lower = uplo == 'L' || uplo == 'l', upper = uplo == 'U' || uplo == 'u';
    if (!lower && !upper) return -1;
    if (batch < 0) return -6;
    if (max_n < 0) return -7;
    if (max_n > BF_VBATCHED_POTRF_NMAX) return BF_ERR_NOT_SUPPORTED;
    if (batch == 0) return BF_SUCCESS;
    if (!n) return -2;
    if (!Aarray) return -3;
    if (!lda) return -4;
    return vb_status(launch_dpotrf_vbatched(n, Aarray, lda, info, batch, max_n, (cudaStream_t)stream, upper ? 1 : 0));
}

extern "C" int bf_dpotrs_vbatched(char uplo, const int* n, const int* nrhs, const double* const* Aarray,
                                  const int* lda, double* const* Barray, const int* ldb, int batch, int max_n,
                                  int max_nrhs, int* dinfo, bf_stream_t stream) {
    const bool lower = uplo == 'L' || uplo == 'l', upper = uplo == 'U' || uplo == 'u';
    if (!lower && !upper) return -1;
    if (batch < 0) return -8;
    if (max_n < 0) return -9;
    if (max_nrhs < 0) return -10;
    if (batch == 0) return BF_SUCCESS;
    if (!n) return -2;
    if (!nrhs) return -3;
    if (!Aarray) return -4;
    if (!lda) return -5;
    if (!Barray) return -6;
    if (!ldb) return -7;
    VPotrsParams p{};
    p.upper = upper; p.n = n; p.nrhs = nrhs; p.A = Aarray; p.lda = lda; p.B = Barray; p.ldb = ldb;
    p.dinfo = dinfo; p.batch = batch; p.max_n = max_n; p.max_nrhs = max_nrhs;
    return vb_status(launch_dpotrs_vbatched(p, (cudaStream_t)stream));
}
