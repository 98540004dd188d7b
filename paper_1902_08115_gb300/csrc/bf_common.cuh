// bf_common.cuh -- device building blocks shared by the batched FP64 kernels.
//
// The paper builds every BLAS/LAPACK kernel from a few shared "inner
// functions" (load, multiply-accumulate over k, scale, edge factorisation,
// store; section 3.2.1).  These are their GPU counterparts: small
// __forceinline__ device functions that the routine kernels compose.
//
// Storage is column-major with a leading dimension (section 2.1): element
// (i, j) of a matrix X with leading dimension ldx is X[i + j * ldx].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bf {

// A batch of matrices: either strided (base + q * stride) or an array of
// per-problem device pointers (arr[q] + off).  `off` lets the blocked
// routines address a sub-matrix of every problem in a pointer-array batch.
struct MatRef {
    const double* base;
    const double* const* arr;
    long long stride;
    long long off;

    __device__ __forceinline__ const double* ptr(long long q) const {
        return arr ? (arr[q] + off) : (base + q * stride);
    }
    __device__ __forceinline__ double* mptr(long long q) const {
        return const_cast<double*>(ptr(q));
    }
};

__host__ __device__ inline MatRef mat_strided(const double* p, long long stride) {
    MatRef r;
    r.base = p;
    r.arr = nullptr;
    r.stride = stride;
    r.off = 0;
    return r;
}

__host__ __device__ inline MatRef mat_array(const double* const* a, long long off) {
    MatRef r;
    r.base = nullptr;
    r.arr = a;
    r.stride = 0;
    r.off = off;
    return r;
}

// Sub-matrix view: element (i0, j0) of every problem.
__host__ __device__ inline MatRef mat_sub(MatRef m, long long i0, long long j0, long long ld) {
    long long d = i0 + j0 * ld;
    if (m.arr) {
        m.off += d;
    } else {
        m.base += d;
    }
    return m;
}

// Scalar modes of C <= alpha * acc + beta * C, chosen on the host so that the
// common cases spend no FP64 instruction on scaling:
//   ACC_ZERO : alpha == 1, beta == 0  -> C = acc            (C not read)
//   ACC_C    : alpha == 1, beta == 1  -> acc starts from C
//   ACC_BC   : alpha == 1, other beta -> acc starts from beta * C
//   ACC_GEN  : other alpha            -> C = alpha * acc + beta * C (C not read if beta == 0)
enum AccMode : int { ACC_ZERO = 0, ACC_C = 1, ACC_BC = 2, ACC_GEN = 3 };

__host__ inline int acc_mode(double alpha, double beta) {
    if (alpha == 1.0) {
        if (beta == 0.0) return ACC_ZERO;
        if (beta == 1.0) return ACC_C;
        return ACC_BC;
    }
    return ACC_GEN;
}

// Store masks of the dgemm kernel (which triangle of C is written).
enum TriMask : int { TRI_NONE = 0, TRI_LOWER = 1, TRI_UPPER = 2, TRI_SLOWER = 3, TRI_SUPPER = 4 };

__host__ __device__ __forceinline__ bool in_tri(int tri, int i, int j) {
    return tri == TRI_NONE || (tri == TRI_LOWER && i >= j) || (tri == TRI_UPPER && i <= j) ||
           (tri == TRI_SLOWER && i > j) || (tri == TRI_SUPPER && i < j);
}

__device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }
__device__ __forceinline__ int imax(int a, int b) { return a > b ? a : b; }

// Read-only global load through the non-coherent path (operands that the
// kernel never writes).
__device__ __forceinline__ double ldg(const double* p) { return __ldg(p); }
// two consecutive doubles from a 16-byte-aligned address, read-only path
__device__ __forceinline__ double2 ldg2(const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); }

}  // namespace bf
