// bf_probe.cu -- launch accounting and the FP64 roofline calibration.
//
// bf_launch_count(): every kernel launch of this library increments one
// host-side counter, so a caller can count the library's launches over a
// region of work.
//
// bf_probe_fp64(): a kernel that issues only FP64 fused multiply-adds in
// the 4x4 register-tile pattern of the routines (16 per iteration, full warps).  Timed by the caller, it
// gives the FP64 FMA throughput of the GPU at its current clocks: the compute
// roof against which the batched routines are placed (every routine here is
// bound by the FP64 pipe, not by memory, for orders >= 8 on this GPU).
#include <atomic>

#include "bf_internal.h"
#include "../../include/bfgpu.h"

namespace bf {

static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

__global__ void __launch_bounds__(256) probe_fp64_kernel(double* out, int iters, double s) {
    // the register-tile pattern of the routines: acc[i][j] += a[i] * b[j] on a 4x4 tile
    // (plain chains a = fma(a, b, c) issue about 17% slower on this GPU)
    double a[4], b[4], acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        a[i] = s + threadIdx.x * 1e-9 + i * 1e-7;
        b[i] = 1.0 - i * 1e-8 - blockIdx.x * 1e-12;
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
    }
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    double r = 0.0;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) r += acc[i][j];
    out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = r;
}

// Variants for the machine-model measurements: `active` lanes of every warp issue the FMAs
// (the others are masked off), `chains` = 0 uses the 4x4 tile pattern, 1 a single dependent
// chain per thread (a = fma(a, b, c)).
__global__ void __launch_bounds__(1024) probe_fp64_ex_kernel(double* out, int iters, int active, int chains) {
    const int lane = threadIdx.x & 31;
    double r = 0.0;
    if (lane < active) {
        if (chains == 0) {
            double a[4], b[4], acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                a[i] = 0.999999 + threadIdx.x * 1e-9 + i * 1e-7;
                b[i] = 1.0 - i * 1e-8 - blockIdx.x * 1e-12;
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
            }
            for (int it = 0; it < iters; it++) {
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) r += acc[i][j];
        } else {
            double a = threadIdx.x * 1e-3, b = 0.999999 - blockIdx.x * 1e-12, c = 0.5;
            for (int it = 0; it < iters; it++) {
#pragma unroll
                for (int u = 0; u < 16; u++) a = fma(a, b, c);
            }
            r = a;
        }
    }
    out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = r;
}

// Other FP64-pipe instruction kinds, each timed like the FMA probe so that their costs can be
// put in DFMA issue slots (kinds as in bf_probe_kind of include/bfgpu.h):
//   0, 1  FP64 tensor-core MMA (DMMA) through mma.sync, shapes m8n8k4 and m16n8k4, four
//         independent accumulators per warp;
//   2..4  sqrt, 1/x and rsqrt of FP64 values, each followed by one FMA (four independent
//         chains per thread: v = fma(op(v), b, c));
//   5     binary32 FMA in the 4x4 register-tile pattern;
//   6     FP64 FMA in the 4x4 register-tile pattern, but only the warps whose index in the CTA is
//         a multiple of 4 issue (the others exit): with 16-warp CTAs, 4 busy warps that share
//         one SM sub-partition if warps are dealt to sub-partitions by index modulo 4.
__device__ __forceinline__ void dmma_m8n8k4(double (&d)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

__device__ __forceinline__ void dmma_m16n8k4(double (&d)[4], double a0, double a1, double b) {
    asm volatile(
        "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0, %1, %2, %3}, {%4, %5}, {%6}, {%0, %1, %2, %3};\n"
        : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
        : "d"(a0), "d"(a1), "d"(b));
}

__global__ void __launch_bounds__(1024) probe_kind_kernel(double* out, int iters, int kind) {
    const double a = 0.999999 + threadIdx.x * 1e-9, b = 1.0 - blockIdx.x * 1e-12;
    double r = 0.0;
    if (kind == 0) {
        double d[4][2] = {};
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int u = 0; u < 4; u++) dmma_m8n8k4(d[u], a + u * 1e-7, b);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) r += d[u][0] + d[u][1];
    } else if (kind == 1) {
        double d[4][4] = {};
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int u = 0; u < 4; u++) dmma_m16n8k4(d[u], a + u * 1e-7, a - u * 1e-7, b);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) r += d[u][0] + d[u][1] + d[u][2] + d[u][3];
    } else if (kind >= 2 && kind <= 4) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = 1.5 + threadIdx.x * 1e-6 + u * 1e-3;
        const double c = 0.75, bb = 0.5;
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const double o = kind == 2 ? sqrt(v[u]) : kind == 3 ? 1.0 / v[u] : rsqrt(v[u]);
                v[u] = fma(o, bb, c);  // stays in [0.75, 1.5]: no special cases
            }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) r += v[u];
    } else if (kind == 6) {
        if ((threadIdx.x >> 5) & 3) return;
        double ta[4], tb[4], acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            ta[i] = a + i * 1e-7;
            tb[i] = b - i * 1e-8;
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
        }
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(ta[i], tb[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) r += acc[i][j];
    } else {
        float fa[4], fb[4], acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            fa[i] = 0.999f + threadIdx.x * 1e-7f + i * 1e-5f;
            fb[i] = 1.0f - i * 1e-6f;
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j] = 0.0f;
        }
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmaf(fa[i], fb[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) r += acc[i][j];
    }
    out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = r;
}

}  // namespace bf

extern "C" int bf_probe_kind(int kind, int blocks, int threads, int iters, double* out, bf_stream_t stream) {
    if (kind < 0 || kind > 6) return -1;
    if (blocks <= 0) return -2;
    if (threads <= 0 || threads > 1024 || threads % 32) return -3;
    if (iters <= 0) return -4;
    if (!out) return -5;
    bf::probe_kind_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(out, iters, kind);
    bf::count_launch();
    return cudaGetLastError() == cudaSuccess ? BF_SUCCESS : BF_ERR_CUDA;
}

extern "C" int bf_probe_fp64_ex(int blocks, int threads, int iters, int active, int chains, double* out,
                                bf_stream_t stream) {
    if (blocks <= 0) return -1;
    if (threads <= 0 || threads > 1024 || threads % 32) return -2;
    if (iters <= 0) return -3;
    if (active < 0 || active > 32) return -4;
    if (chains < 0 || chains > 1) return -5;
    if (!out) return -6;
    bf::probe_fp64_ex_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(out, iters, active, chains);
    bf::count_launch();
    return cudaGetLastError() == cudaSuccess ? BF_SUCCESS : BF_ERR_CUDA;
}

extern "C" unsigned long long bf_launch_count(void) {
    return bf::g_launches.load(std::memory_order_relaxed);
}

extern "C" int bf_probe_fp64(int blocks, int iters, double* out, bf_stream_t stream) {
    if (blocks <= 0) return -1;
    if (iters <= 0) return -2;
    if (!out) return -3;
    bf::probe_fp64_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(out, iters, 0.999999);
    bf::count_launch();
    return cudaGetLastError() == cudaSuccess ? BF_SUCCESS : BF_ERR_CUDA;
}
