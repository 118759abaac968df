// Vectorised access helpers and the coefficient pass of the low-rank
// P / P^{-1} apply (Eq. RYPreconditioner in Woodbury form), shared by the
// standalone apply and the fused prox kernels.
#pragma once

#include "internal.cuh"

namespace nys {
namespace {

template <class T> struct Vec16;
template <> struct Vec16<__nv_bfloat16> { static constexpr int n = 8; };
template <> struct Vec16<float> { static constexpr int n = 4; };
template <> struct Vec16<double> { static constexpr int n = 2; };

// 16-byte loads unpacked in registers (bf16 -> f32 is a 16-bit shift)
template <class TU, class TA, int V>
__device__ __forceinline__ void load_vec(const TU* p, TA (&v)[V]);

template <>
__device__ __forceinline__ void load_vec<__nv_bfloat16, float, 8>(const __nv_bfloat16* p, float (&v)[8]) {
    const uint4 r = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[2 * k] = __uint_as_float(w[k] << 16);
        v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
}
template <>
__device__ __forceinline__ void load_vec<float, float, 4>(const float* p, float (&v)[4]) {
    const float4 r = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = r.x, v[1] = r.y, v[2] = r.z, v[3] = r.w;
}
template <>
__device__ __forceinline__ void load_vec<double, double, 2>(const double* p, double (&v)[2]) {
    const double2 r = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = r.x, v[1] = r.y;
}

// L2 eviction priorities for loads of U (PTX createpolicy + ld.L2::cache_hint):
// evict_last for the columns meant to stay in L2 across applications,
// evict_first for the columns that stream through.
struct L2Pol {
    uint64_t last, first;
};
__device__ __forceinline__ L2Pol make_l2_pol() {
    L2Pol p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p.last));
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p.first));
    return p;
}
template <class TU, class TA, int V>
__device__ __forceinline__ void load_vec_pol(const TU* p, TA (&v)[V], uint64_t pol);
template <>
__device__ __forceinline__ void load_vec_pol<__nv_bfloat16, float, 8>(const __nv_bfloat16* p, float (&v)[8],
                                                                     uint64_t pol) {
    uint32_t w[4];
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
                 : "l"(p), "l"(pol));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[2 * k] = __uint_as_float(w[k] << 16);
        v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
}
template <>
__device__ __forceinline__ void load_vec_pol<float, float, 4>(const float* p, float (&v)[4], uint64_t pol) {
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "l"(p), "l"(pol));
}
template <>
__device__ __forceinline__ void load_vec_pol<double, double, 2>(const double* p, double (&v)[2], uint64_t pol) {
    asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v[0]), "=d"(v[1]) : "l"(p), "l"(pol));
}

// 128-bit shared-memory loads of V compute-type values (V * sizeof(TA) is a
// multiple of 16 bytes)
template <class TA, int V>
__device__ __forceinline__ void lds_vec(const TA* p, TA (&v)[V]);
template <>
__device__ __forceinline__ void lds_vec<float, 8>(const float* p, float (&v)[8]) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
}
template <>
__device__ __forceinline__ void lds_vec<float, 4>(const float* p, float (&v)[4]) {
    const float4 a = reinterpret_cast<const float4*>(p)[0];
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
}
template <>
__device__ __forceinline__ void lds_vec<double, 2>(const double* p, double (&v)[2]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    v[0] = a.x, v[1] = a.y;
}

// w[j] = sum_c partT[j * nb + c] (column-major partials: column j's chunk sums
// are contiguous), one warp per column, all of a warp's columns loaded before
// they are summed (four at a time), fixed order.  Ends with __syncthreads().
template <class TA>
__device__ __forceinline__ void reduce_partials_t(const TA* __restrict__ partT, int nb, int le, TA* w) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j0 = warp; j0 < le; j0 += 4 * nw) {
        TA acc[4] = {TA(0), TA(0), TA(0), TA(0)};
        for (int c0 = 0; c0 < nb; c0 += 32 * 8) {
            TA v[4][8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = j0 + q * nw;
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int c = c0 + r * 32 + lane;
                    v[q][r] = (j < le && c < nb) ? __ldcg(partT + (size_t)j * nb + c) : TA(0);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int r = 0; r < 8; ++r) acc[q] += v[q][r];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const TA sq = warp_sum(acc[q]);
            const int j = j0 + q * nw;
            if (lane == 0 && j < le) w[j] = sq;
        }
    }
    __syncthreads();
}

// coef[r] = inverse ? sum_k M[r][k] w[k] : d[r] w[r] for r in [r0, r1), one
// warp per row
template <class TA, class TM>
__device__ __forceinline__ void coef_rows(const TA* w, int le, int ldm, int inverse, const TM* __restrict__ M,
                                          const TM* __restrict__ d, int r0, int r1, TA* __restrict__ coef) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = r0 + warp; r < r1; r += nw) {
        TA s;
        if (inverse) {
            s = TA(0);
            for (int k = lane; k < le; k += 32) s = fma((TA)M[(size_t)r * ldm + k], w[k], s);
            s = warp_sum(s);
        } else {
            s = (TA)d[r] * w[r];
        }
        if (lane == 0) coef[r] = s;
    }
}

// coef[b][r] for the 32 rows r of this CTA (batch b = blockIdx.y); every CTA
// rebuilds w from the column-major partials part[b][j][c].  Dynamic shared
// memory: le TA.  For small le (the rebuild is le x nb loads per CTA).
template <class TA, class TM>
__global__ void __launch_bounds__(256) coef_vec_kernel(const TA* __restrict__ part, int nb, int le, int ldm,
                                                       int inverse, const TM* __restrict__ M,
                                                       const TM* __restrict__ d, TA* __restrict__ coef) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TA* w = reinterpret_cast<TA*>(smem_raw);
    const int b = blockIdx.y;
    reduce_partials_t<TA>(part + (size_t)b * nb * le, nb, le, w);
    const int r0 = blockIdx.x * 32;
    coef_rows<TA, TM>(w, le, ldm, inverse, M, d, r0, min(le, r0 + 32), coef + (size_t)b * le);
}

// Large le, two passes spread over many CTAs.  reduce_cols: w[b][j] =
// sum_c part[b][j][c], one warp per column (8 per CTA); mw: coef[b][r] =
// inverse ? sum_k M[r][k] w[b][k] : d[r] w[b][r], one warp per row.
// (stop: inside the dual iteration of the prox, a skipped step does nothing)
template <class TA>
__global__ void __launch_bounds__(256) reduce_cols_kernel(const TA* __restrict__ part, int nb, int le,
                                                          TA* __restrict__ w, DualStop stop) {
    pdl_enter();
    if (dual_skip(stop)) return;
    const int j = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31, b = blockIdx.y;
    if (j >= le) return;
    const TA* p = part + ((size_t)b * le + j) * nb;
    TA a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = TA(0);
    for (int c0 = 0; c0 < nb; c0 += 256) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = c0 + q * 32 + lane;
            if (c < nb) a[q] += p[c];
        }
    }
    TA s = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    s = warp_sum(s);
    if (lane == 0) w[(size_t)b * le + j] = s;
}

template <class TA, class TM>
__global__ void __launch_bounds__(256) mw_kernel(const TM* __restrict__ M, int ldm, int inverse,
                                                 const TM* __restrict__ d, const TA* __restrict__ w, int le,
                                                 TA* __restrict__ coef, DualStop stop) {
    pdl_enter();
    if (dual_skip(stop)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TA* ws = reinterpret_cast<TA*>(smem_raw);
    const int b = blockIdx.y;
    for (int k = threadIdx.x; k < le; k += blockDim.x) ws[k] = w[(size_t)b * le + k];
    __syncthreads();
    coef_rows<TA, TM>(ws, le, ldm, inverse, M, d, blockIdx.x * 8, min(le, blockIdx.x * 8 + 8), coef + (size_t)b * le);
}

// c = M w (or d .* w) from column-major partials, choosing the one-kernel
// path for small le and the two-kernel path otherwise
template <class TA, class TM>
int coef_run(nys_ctx* ctx, const TA* part, int nb, int le, int ldm, int inverse, const TM* M, const TM* d,
             TA* coef, int batch, TA* wbuf = nullptr, DualStop stop = {}) {
    cudaStream_t s = ctx->stream;
    if (le <= 64 || !wbuf) {
        NYS_CK(ctx, launch_pdl(coef_vec_kernel<TA, TM>, dim3((le + 31) / 32, batch), 256, le * sizeof(TA), s, part,
                               nb, le, ldm, inverse, M, d, coef));
        NYS_LAUNCH_CK(ctx);
        return NYS_OK;
    }
    NYS_CK(ctx, launch_pdl(reduce_cols_kernel<TA>, dim3((le + 7) / 8, batch), 256, 0, s, part, nb, le, wbuf, stop));
    NYS_LAUNCH_CK(ctx);
    NYS_CK(ctx, launch_pdl(mw_kernel<TA, TM>, dim3((le + 7) / 8, batch), 256, le * sizeof(TA), s, M, ldm, inverse, d,
                           wbuf, le, coef, stop));
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

// End of a 1-D partial-sum pass whose CTAs wrote column-major partials
// partT[j * gridDim.x + blockIdx.x]: the last CTA to arrive (counted on
// *counter, zero before the launch and reset here) reduces them and writes
// coef = M w (one thread per row).  No CTA waits for another.  sm: le TA,
// plus le * le TA when le <= 64 (M is staged in shared memory).
template <class TA, class TM>
__device__ __forceinline__ void last_cta_coef_t(const TA* partT, int le, int ldm, const TM* __restrict__ M,
                                                TA* __restrict__ coef, unsigned* counter, TA* sm) {
    __shared__ unsigned is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    reduce_partials_t<TA>(partT, gridDim.x, le, sm);
    if (le <= 64) {
        // stage the le x le block of M (coalesced, one round of loads)
        TA* Ms = sm + le;
        for (int e = threadIdx.x; e < le * le; e += blockDim.x) Ms[e] = (TA)M[(size_t)(e / le) * ldm + e % le];
        __syncthreads();
        for (int r = threadIdx.x; r < le; r += blockDim.x) {
            TA a = TA(0);
            for (int k = 0; k < le; ++k) a = fma(Ms[r * le + k], sm[k], a);
            coef[r] = a;
        }
    } else {
        for (int r = threadIdx.x; r < le; r += blockDim.x) {
            const TM* mr = M + (size_t)r * ldm;
            TA a[4] = {TA(0), TA(0), TA(0), TA(0)};
            int k = 0;
            for (; k + 4 <= le; k += 4) {
#pragma unroll
                for (int q = 0; q < 4; ++q) a[q] = fma((TA)mr[k + q], sm[k + q], a[q]);
            }
            for (; k < le; ++k) a[0] = fma((TA)mr[k], sm[k], a[0]);
            coef[r] = (a[0] + a[1]) + (a[2] + a[3]);
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// out = z + sign * U c, or with base: out = base + scale (z + sign U c).  A CTA
// owns 32 V PV pixels (PV 16-byte vectors per lane); its 8 warps split the
// columns, NQ columns per round, and their partial sums meet in shared memory
template <class TU, class TZ, class TA, int NQ = 4, int PV = 1>
__global__ void __launch_bounds__(256) uc_vec_kernel(const TU* __restrict__ U, const TZ* __restrict__ z, int64_t N,
                                                     int ell, const TA* __restrict__ coef, TA sign,
                                                     TZ* __restrict__ out, const TZ* __restrict__ base, TA scale,
                                                     int keep, DualStop stop) {
    pdl_enter();
    constexpr int V = Vec16<TU>::n;
    constexpr int P = 32 * V * PV;
    if (dual_skip(stop)) {
        if (stop.copy)
            for (int p = threadIdx.x; p < P; p += blockDim.x) {
                const int64_t ii = (int64_t)blockIdx.x * P + p;
                if (ii < N) {
                    const size_t o = (size_t)blockIdx.y * N + ii;
                    out[o] = reinterpret_cast<const TZ*>(stop.copy)[o];
                }
            }
        return;
    }
    const L2Pol pol = make_l2_pol();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TA* c = reinterpret_cast<TA*>(smem_raw);
    TA* red = c + ((ell + 3) & ~3);            // [8][P]
    const int b = blockIdx.y;
    for (int j = threadIdx.x; j < ell; j += blockDim.x) c[j] = coef[(size_t)b * ell + j];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    TA acc[PV][V];
#pragma unroll
    for (int v = 0; v < PV; ++v)
#pragma unroll
        for (int k = 0; k < V; ++k) acc[v][k] = TA(0);
    // NQ columns (j, j + 8, ...) per round, loads predicated, so a small
    // active set still has all its loads in flight at once
    for (int j = warp; j < ell; j += 8 * NQ) {
        TA u[NQ][PV][V];
        TA cq[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int jq = j + 8 * q;
            cq[q] = jq < ell ? c[jq] : TA(0);
#pragma unroll
            for (int v = 0; v < PV; ++v) {
                const int64_t i = (int64_t)blockIdx.x * P + (v * 32 + lane) * V;
                if (jq < ell && i < N)
                    load_vec_pol<TU, TA, V>(U + (size_t)jq * N + i, u[q][v], jq < keep ? pol.last : pol.first);
                else
#pragma unroll
                    for (int k = 0; k < V; ++k) u[q][v][k] = TA(0);
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int v = 0; v < PV; ++v)
#pragma unroll
                for (int k = 0; k < V; ++k) acc[v][k] = fma(u[q][v][k], cq[q], acc[v][k]);
    }
#pragma unroll
    for (int v = 0; v < PV; ++v)
#pragma unroll
        for (int k = 0; k < V; ++k) red[warp * P + (v * 32 + lane) * V + k] = acc[v][k];
    __syncthreads();
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const int64_t ii = (int64_t)blockIdx.x * P + p;
        if (ii >= N) continue;
        TA s = TA(0);
#pragma unroll
        for (int w = 0; w < 8; ++w) s += red[w * P + p];
        const size_t o = (size_t)b * N + ii;
        const TA v = (TA)ldf(z + o) + sign * s;
        stf(out + o, base ? (TA)ldf(base + o) + scale * v : v);
    }
}

}  // namespace
}  // namespace nys
