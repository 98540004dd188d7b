// bf_probe.cu -- launch accounting and the FP64 roofline calibration.
//
// bf_launch_count(): every kernel launch of this library increments one
// host-side counter, so a caller can count the library's launches over a
// region of work.
//
// bf_probe_fp64(): a kernel that issues only independent FP64 fused
// multiply-adds (8 chains per thread, full warps).  Timed by the caller, it
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
    double a[8];
#pragma unroll
    for (int i = 0; i < 8; i++) a[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) a[i] = fma(a[i], s, 0.5);
    }
    double r = 0.0;
#pragma unroll
    for (int i = 0; i < 8; i++) r += a[i];
    out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = r;
}

}  // namespace bf

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
