// Periodic difference stencils of the regularisers (Appendix A): L^T Q at one
// pixel for the first differences (anisotropic TV) and the second differences
// (Hessian), shared by the prox kernels and the unrolled-solve kernels.
#pragma once

#include "internal.cuh"

namespace nys {

template <class T>
__device__ __forceinline__ T at(const T* p, int i, int j, int n1, int n2) {
    return p[(size_t)pmod(i, n1) * n2 + pmod(j, n2)];
}

// L^T Q at pixel (i, j)
template <class T, int REG>
__device__ __forceinline__ typename Comp<T>::type lt_q(const T* __restrict__ Q, int i, int j, int n1, int n2) {
    using TC = typename Comp<T>::type;
    const size_t N = (size_t)n1 * n2;
    if (REG == NYS_REG_TV) {
        const T* q1 = Q;
        const T* q2 = Q + N;
        return (TC)at(q1, i, j, n1, n2) - (TC)at(q1, i + 1, j, n1, n2) + (TC)at(q2, i, j, n1, n2) -
               (TC)at(q2, i, j + 1, n1, n2);
    } else {
        const T* q11 = Q;
        const T* q12 = Q + N;
        const T* q22 = Q + 2 * N;
        const TC a11 = (TC)at(q11, i - 1, j, n1, n2) - TC(2) * (TC)at(q11, i, j, n1, n2) + (TC)at(q11, i + 1, j, n1, n2);
        const TC a22 = (TC)at(q22, i, j - 1, n1, n2) - TC(2) * (TC)at(q22, i, j, n1, n2) + (TC)at(q22, i, j + 1, n1, n2);
        const TC a12 = TC(0.25) * ((TC)at(q12, i + 1, j + 1, n1, n2) - (TC)at(q12, i + 1, j - 1, n1, n2) -
                                   (TC)at(q12, i - 1, j + 1, n1, n2) + (TC)at(q12, i - 1, j - 1, n1, n2));
        return a11 + TC(2) * a12 + a22;
    }
}

}  // namespace nys
