// One-CTA in-place Cholesky shared by the factor and the Newton prox.
#pragma once
#include "internal.cuh"

namespace nys {

// in-place lower Cholesky of an n x n row-major matrix by one CTA; returns
// false (uniformly) if a pivot is not positive.  `flag` is shared memory.
__device__ __forceinline__ bool block_cholesky(double* A, int n, int* flag) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            const double d = A[(size_t)k * n + k];
            if (!(d > 0.0) || !isfinite(d)) *flag = 1;
            else A[(size_t)k * n + k] = sqrt(d);
        }
        __syncthreads();
        if (*flag) return false;
        const double dk = A[(size_t)k * n + k];
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[(size_t)i * n + k] /= dk;
        __syncthreads();
        const int m = n - k - 1;
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
            const int i = k + 1 + t / m, j = k + 1 + t % m;
            if (j <= i) A[(size_t)i * n + j] -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int i = t / n, j = t % n;
        if (j > i) A[t] = 0.0;
    }
    __syncthreads();
    return true;
}

}  // namespace nys
