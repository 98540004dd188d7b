// bf_stage.cuh -- staging of a CTA's small problems through shared memory.
//
// The packed forms of the paper (section 2.2, 'B'/'C') copy operands into a buffer laid out
// for the inner kernel.  For problems of a few rows, the GPU's inner kernel is one thread per
// problem, and what it needs is (a) global traffic that is coalesced and vectorised -- the
// CTA's problems are usually one contiguous run of memory, read as 16-byte pieces by
// consecutive threads -- and (b) a shared-memory layout where thread qq reads its element e
// at s[e * ST + qq]: consecutive threads touch consecutive words.  ST = threads + 1 staggers
// the banks of the staging stores, whose consecutive lanes write consecutive elements of one
// problem.
#pragma once

#include "bf_common.cuh"

namespace bf {

// The CTA's nq problems of a batch, rows x cols each (leading dimension ld), are one
// contiguous, 16-byte-aligned run of an even number of doubles.
__device__ __forceinline__ bool stage_contiguous(const MatRef& X, int rows, int cols, int ld, long long q0) {
    const int per = rows * cols;
    return !X.arr && X.stride == per && ld == rows && (per & 1) == 0 &&
           (reinterpret_cast<uintptr_t>(X.ptr(q0)) & 15u) == 0;
}

// One element copied from global to shared memory without passing through registers.
__device__ __forceinline__ void stage_copy8(double* dst, const double* src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(src) : "memory");
}

// Waits for this thread's stage_in copies; a CTA barrier must follow before other threads
// read the staged problems.
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// s[e * ST + qq] = X_(q0+qq)(i, j), e = i + j rows (trans: X_(q0+qq)(j, i)); nq problems.  The
// copies are asynchronous, all of a thread's in flight at once: complete them with stage_wait().
__device__ __forceinline__ void stage_in(const MatRef& X, int rows, int cols, int ld, bool trans, long long q0,
                                         int nq, double* s, int ST) {
    const int per = rows * cols;
    const int T = blockDim.x;
    if (!trans && stage_contiguous(X, rows, cols, ld, q0)) {
        const double* base = X.ptr(q0);
        for (int t = threadIdx.x; 2 * t < nq * per; t += T) {
            const int f = 2 * t, qq = f / per, e = f - qq * per;
            stage_copy8(s + e * ST + qq, base + f);
            stage_copy8(s + (e + 1) * ST + qq, base + f + 1);
        }
        return;
    }
    // element f = (problem qq, column j, row i), rows fastest, stepped by T without divisions
    int qq = threadIdx.x / per;
    int j = (threadIdx.x - qq * per) / rows, i = threadIdx.x - qq * per - j * rows;
    const int dq = T / per, dj = (T - dq * per) / rows, di = T - dq * per - dj * rows;
    for (int f = threadIdx.x; f < nq * per; f += T) {
        const double* x = X.ptr(q0 + qq);
        stage_copy8(s + (i + j * rows) * ST + qq, trans ? x + j + (long long)i * ld : x + i + (long long)j * ld);
        qq += dq;
        i += di;
        j += dj;
        if (i >= rows) {
            i -= rows;
            j++;
        }
        if (j >= cols) {
            j -= cols;
            qq++;
        }
    }
}

// The inverse: X_(q0+qq)(i, j) = s[e * ST + qq] for every element (trans: X(j, i)), or only for
// the elements where keep(i, j) holds.
template <class Keep>
__device__ __forceinline__ void stage_out(const MatRef& X, int rows, int cols, int ld, bool trans, long long q0,
                                          int nq, const double* s, int ST, bool all, const Keep& keep) {
    const int per = rows * cols;
    const int T = blockDim.x;
    if (all && !trans && stage_contiguous(X, rows, cols, ld, q0)) {
        double* base = X.mptr(q0);
        for (int t = threadIdx.x; 2 * t < nq * per; t += T) {
            const int f = 2 * t, qq = f / per, e = f - qq * per;
            reinterpret_cast<double2*>(base)[t] = make_double2(s[e * ST + qq], s[(e + 1) * ST + qq]);
        }
        return;
    }
    int qq = threadIdx.x / per;
    int j = (threadIdx.x - qq * per) / rows, i = threadIdx.x - qq * per - j * rows;
    const int dq = T / per, dj = (T - dq * per) / rows, di = T - dq * per - dj * rows;
    for (int f = threadIdx.x; f < nq * per; f += T) {
        if (all || keep(i, j)) {
            double* x = X.mptr(q0 + qq);
            const double v = s[(i + j * rows) * ST + qq];
            if (trans) x[j + (long long)i * ld] = v;
            else x[i + (long long)j * ld] = v;
        }
        qq += dq;
        i += di;
        j += dj;
        if (i >= rows) {
            i -= rows;
            j++;
        }
        if (j >= cols) {
            j -= cols;
            qq++;
        }
    }
}

}  // namespace bf
