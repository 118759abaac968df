// Two steps of the right-looking panel Cholesky that the cluster kernels
// (chol_cluster.cu in float64, jacobi_cluster.cu in float32) share.  Panels
// are at most 16 columns wide; the upper factor R (A = R^T R) is stored by
// columns, R(i, j) at col(j)[i].
#pragma once

#include <cuda_runtime.h>

namespace nys {

// r = sqrt(d) and ri = 1 / r: correctly rounded in float64; in float32 from
// one hardware reciprocal square root (a few ulp, the accuracy the float32
// eigensolver's rotations work at), which shortens the block's dependent
// chain by a square root and a division per column
__device__ __forceinline__ void pivot_root(double d, double& r, double& ri) {
    r = sqrt(d);
    ri = 1.0 / r;
}
__device__ __forceinline__ void pivot_root(float d, float& r, float& ri) {
    ri = rsqrtf(d);
    r = d * ri;
}

// The b x b diagonal block of the panel starting at p0 (b <= 16), factored in
// place by one warp: lane c keeps column c of the block in registers, row t
// of R is scaled by the pivot's reciprocal and broadcast lane by lane by
// shuffles.  Only the upper triangle (row <= column) is read and written.
// Returns false, identically in every lane, on a pivot that is not positive
// and finite (nothing is written back then).
template <class T, int NB, class ColFn>
__device__ __forceinline__ bool warp_chol_block_nb(ColFn col, int p0, int b) {
    const int lane = threadIdx.x & 31;
    T a[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) a[i] = (lane < b && i <= lane) ? col(lane)[p0 + i] : T(0);
    bool ok = true;
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        if (t < b) {
            const T d = __shfl_sync(0xffffffffu, a[t], t);   // the same value in every lane
            if (!(d > T(0)) || !isfinite(d)) {
                ok = false;
                break;
            }
            T r, ri;
            pivot_root(d, r, ri);
            if (lane == t) a[t] = r;
            else if (lane > t) a[t] *= ri;   // R(t, lane)
            // R(i, c) -= R(t, i) R(t, c) for t < i <= c; R(t, i) from lane i
#pragma unroll
            for (int i = t + 1; i < NB; ++i) {
                const T rti = __shfl_sync(0xffffffffu, a[t], i);
                if (lane >= i) a[i] -= rti * a[t];
            }
        }
    }
    if (ok && lane < b) {
        T* c = col(lane);
#pragma unroll
        for (int i = 0; i < NB; ++i)
            if (i <= lane) c[p0 + i] = a[i];
    }
    return ok;
}

// Unrolled to 8 or 16 columns: the float64 pipe is narrow, so no
// predicated-off arithmetic for narrow panels.
template <class T, class ColFn>
__device__ __forceinline__ bool warp_chol_block(ColFn col, int p0, int b) {
    return b <= 8 ? warp_chol_block_nb<T, 8>(col, p0, b) : warp_chol_block_nb<T, 16>(col, p0, b);
}

// The panel's rows of one later column: solve R_PP^T x = g by forward
// substitution, g = c[p0 .. p0 + b) in place; R_PP staged column by column,
// stage[k * b + i] = R(p0 + i, p0 + k).  The column stays in registers.
// The reciprocals of the diagonal are formed first, off the dependent chain.
template <class T, int NB>
__device__ __forceinline__ void panel_forward_subst_nb(T* c, const T* stage, int p0, int b) {
    T x[NB], rd[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        x[i] = i < b ? c[p0 + i] : T(0);
        rd[i] = i < b ? T(1) / stage[i * b + i] : T(0);
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        if (i < b) {
            T acc = x[i];
#pragma unroll
            for (int q = 0; q < i; ++q) acc -= stage[i * b + q] * x[q];
            x[i] = acc * rd[i];
        }
    }
#pragma unroll
    for (int i = 0; i < NB; ++i)
        if (i < b) c[p0 + i] = x[i];
}

template <class T>
__device__ __forceinline__ void panel_forward_subst(T* c, const T* stage, int p0, int b) {
    if (b <= 8) panel_forward_subst_nb<T, 8>(c, stage, p0, b);
    else panel_forward_subst_nb<T, 16>(c, stage, p0, b);
}

}  // namespace nys
