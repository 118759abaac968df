// Algorithm 1 (Nystrom approximation) and the preconditioner of
// Eq. (RYPreconditioner) in its Sec. III-B form P = I + Ubar Ubar^T.
//
// nys_sketch   steps 1-2: Omega from Philox4x32-10 + Box-Muller, Y = Phi Omega
//              through the batched operator (all ell probes in one launch).
// nys_factor   steps 3-8, reorganised so the tall N x ell data is read twice:
//                G2 = [Omega | Y]^T [Omega | Y]            (one Gram pass)
//                v  = eps sqrt(trace(Omega^T Omega))        (step 3)
//                C  = chol(sym(Omega^T Y) + v Omega^T Omega)   (steps 4-5)
//                H  = Y_v^T Y_v from the blocks of G2
//                G  = C^{-1} H C^{-T}  = B^T B for B = Y_v C^{-T}   (step 6)
//                G  = V S^2 V^T                             (step 7, eig of B^T B)
//                U  = B V S^{-1} = (Y + v Omega) (C^{-T} V S^{-1})  (one GEMM pass)
//                S_hat = max(0, S^2 - v)                    (step 8)
//              In exact arithmetic this is Algorithm 1's thin SVD of B.
// precond      weights d_i, K = U^T U of the stored U, and
//              M = diag(sqrt d) (I + Ubar^T Ubar)^{-1} diag(sqrt d), so that
//              P^{-1} z = z - U M U^T z is the exact inverse of P z = z + U diag(d) U^T z.
#include "internal.cuh"
#include "vec.cuh"

#include <cmath>
#include <type_traits>
#include <mutex>

namespace nys {

int launch_small_gemm(nys_ctx* ctx, const double* A, int ta, const double* B, int tb, int m, int n, int k,
                      const double* colscale, double* C);
int sym_eig(nys_ctx* ctx, const double* G, int ell, bool use_f32, const double* info, void* work, double* Vout,
            double* S_hat, double* scale, int* sweeps_dev);
__global__ void shift_chol_kernel(const double* __restrict__ G2, int ell, double eps, int max_retries,
                                  double* __restrict__ C, double* __restrict__ info);
__global__ void form_H_kernel(const double* __restrict__ G2, int ell, const double* __restrict__ info,
                              double* __restrict__ H);
__global__ void tri_inv_kernel(const double* __restrict__ C, double* __restrict__ X, int n);
__global__ void weights_kernel(const double* __restrict__ S_hat, int ell, double mu, int sqrt_shift,
                               double* __restrict__ d, double* __restrict__ sqd, float* __restrict__ d32);
__global__ void form_A_kernel(const double* __restrict__ K, int ldk, const double* __restrict__ sqd, int eff,
                              double* __restrict__ A);
__global__ void chol_kernel(double* __restrict__ A, int n, double* __restrict__ info);
__global__ void form_M_kernel(const double* __restrict__ Ainv, const double* __restrict__ sqd, int ell, int eff,
                              double* __restrict__ M, float* __restrict__ M32);

namespace {

// ------------------------------------------------------------ Philox ----
struct P4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ P4 philox4x32_10(P4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = P4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    }
    return c;
}

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1) {
    const float u0 = ((float)(a >> 9) + 0.5f) * 1.1920928955078125e-7f;   // 2^-23
    const float u1 = ((float)(b >> 9) + 0.5f) * 1.1920928955078125e-7f;
    const float rho = sqrtf(-2.0f * logf(u0));
    float s, c;
    sincospif(2.0f * u1, &s, &c);
    z0 = rho * c;
    z1 = rho * s;
}
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, double& z0, double& z1) {
    const double u0 = ((double)(a >> 9) + 0.5) * 1.1920928955078125e-7;
    const double u1 = ((double)(b >> 9) + 0.5) * 1.1920928955078125e-7;
    const double rho = sqrt(-2.0 * log(u0));
    double s, c;
    sincospi(2.0 * u1, &s, &c);
    z0 = rho * c;
    z1 = rho * s;
}

// out[e - first] for first <= e < first + total: element e of the generator's
// stream (Philox block e / 4, entry e mod 4)
template <class T, class TC>
__global__ void omega_kernel(T* __restrict__ out, int64_t first, int64_t total, uint64_t seed) {
    const int64_t b0 = first / 4, b1 = (first + total + 3) / 4;
    const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    for (int64_t b = b0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < b1;
         b += (int64_t)gridDim.x * blockDim.x) {
        const P4 x = philox4x32_10(P4{(uint32_t)(b & 0xffffffffu), (uint32_t)((uint64_t)b >> 32), 0u, 0u}, k0, k1);
        TC z[4];
        box_muller(x.x, x.y, z[0], z[1]);
        box_muller(x.z, x.w, z[2], z[3]);
        const int64_t e0 = 4 * b;
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (e0 + r >= first && e0 + r < first + total) stf(out + (e0 + r - first), z[r]);
    }
}

// --------------------------------------------------- P / P^{-1} apply ---
constexpr int PCH = 1024;   // pixels per partial-sum block

// part[b][j] = sum_{i in chunk b} U[j][i] z[i]
template <class TU, class TZ, class TA>
__global__ void __launch_bounds__(256) utz_kernel(const TU* __restrict__ U, const TZ* __restrict__ z, int64_t N,
                                                  int ell, TA* __restrict__ part) {
    __shared__ TA zs[PCH];
    const int64_t i0 = (int64_t)blockIdx.x * PCH;
    const int nb = gridDim.x;
    const TZ* zb = z + (size_t)blockIdx.y * N;
    for (int t = threadIdx.x; t < PCH; t += blockDim.x) zs[t] = (i0 + t < N) ? (TA)ldf(zb + i0 + t) : TA(0);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int cnt = (int)(N - i0 < (int64_t)PCH ? N - i0 : (int64_t)PCH);
    for (int j = warp; j < ell; j += nw) {
        const TU* uj = U + (size_t)j * N + i0;
        TA s = TA(0);
        for (int t = lane; t < cnt; t += 32) s = fma((TA)ldf(uj + t), zs[t], s);
        s = warp_sum(s);
        if (lane == 0) part[((size_t)blockIdx.y * nb + blockIdx.x) * ell + j] = s;
    }
}

// coef[b][r] = inverse ? sum_k M[r][k] w[k] : d[r] w[r],  w = sum over partial
// blocks; M has leading dimension ldm >= ell
template <class TA, class TM>
__global__ void __launch_bounds__(256) coef_kernel(const TA* __restrict__ part, int nb, int ell, int ldm,
                                                   int inverse, const TM* __restrict__ M, const TM* __restrict__ d,
                                                   TA* __restrict__ coef) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* w = reinterpret_cast<double*>(smem_raw);
    const int b = blockIdx.y;
    const TA* pb = part + (size_t)b * nb * ell;
    for (int j = threadIdx.x; j < ell; j += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nb; ++k) s += (double)pb[(size_t)k * ell + j];
        w[j] = s;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int r0 = blockIdx.x * 32;
    for (int r = r0 + warp; r < min(ell, r0 + 32); r += nw) {
        double s;
        if (inverse) {
            s = 0.0;
            for (int k = lane; k < ell; k += 32) s += (double)M[(size_t)r * ldm + k] * w[k];
            s = warp_sum(s);
        } else {
            s = (double)d[r] * w[r];
        }
        if (lane == 0) coef[(size_t)b * ell + r] = (TA)s;
    }
}

// out[i] = z[i] + sign * sum_j U[j][i] coef[j]
template <class TU, class TZ, class TA>
__global__ void __launch_bounds__(256) uc_kernel(const TU* __restrict__ U, const TZ* __restrict__ z, int64_t N,
                                                 int ell, const TA* __restrict__ coef, TA sign, TZ* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TA* c = reinterpret_cast<TA*>(smem_raw);
    const int b = blockIdx.y;
    for (int j = threadIdx.x; j < ell; j += blockDim.x) c[j] = coef[(size_t)b * ell + j];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        TA s = TA(0);
        for (int j = 0; j < ell; ++j) s = fma((TA)ldf(U + (size_t)j * N + i), c[j], s);
        const size_t o = (size_t)b * N + i;
        stf(out + o, (TA)ldf(z + o) + sign * s);
    }
}

// ---- vectorised fast path (N a multiple of the 16-byte vector width) ----
// Both passes stream U once with 16-byte loads (8 bf16, 4 f32 or 2 f64 per
// lane) and are sized to put several CTAs on every SM.
constexpr int VCH = 2048;    // pixels per partial-sum chunk

// grid (chunks, column groups): part[b][j][chunk] = sum_{i in chunk} U[j][i] z[i]
// (column-major per batch image: a column's chunk sums are contiguous)
template <class TU, class TZ, class TA>
__global__ void __launch_bounds__(256) utz_vec_kernel(const TU* __restrict__ U, const TZ* __restrict__ z, int64_t N,
                                                      int ell, int jper, TA* __restrict__ part, int keep) {
    pdl_enter();
    const L2Pol l2p = make_l2_pol();
    constexpr int V = Vec16<TU>::n;
    __shared__ __align__(16) TA zs[VCH];
    const int64_t i0 = (int64_t)blockIdx.x * VCH;
    const int nchunk = gridDim.x;
    const TZ* zb = z + (size_t)blockIdx.z * N;
    for (int t = threadIdx.x; t < VCH; t += blockDim.x) zs[t] = (i0 + t < N) ? (TA)ldf(zb + i0 + t) : TA(0);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j0 = blockIdx.y * jper, j1 = min(ell, j0 + jper);
    const int cnt = (int)(N - i0 < (int64_t)VCH ? N - i0 : (int64_t)VCH);   // multiple of V
    for (int j = j0 + warp; j < j1; j += 8) {
        const TU* uj = U + (size_t)j * N + i0;
        const uint64_t pol = j < keep ? l2p.last : l2p.first;
        TA s = TA(0);
        if (cnt == VCH) {
            // full chunk: the trip count is a compile-time constant, so all of a
            // column's 16-byte loads are issued before the FMAs consume them
            constexpr int T = VCH / (32 * V);
            constexpr int G = T < 8 ? T : 8;
#pragma unroll
            for (int t0 = 0; t0 < T; t0 += G) {
                TA u[G][V];
#pragma unroll
                for (int q = 0; q < G; ++q) load_vec_pol<TU, TA, V>(uj + ((t0 + q) * 32 + lane) * V, u[q], pol);
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    const int t = ((t0 + q) * 32 + lane) * V;
                    TA zv[V];
                    lds_vec<TA, V>(zs + t, zv);
#pragma unroll
                    for (int k = 0; k < V; ++k) s = fma(u[q][k], zv[k], s);
                }
            }
            s = warp_sum(s);
            if (lane == 0) part[((size_t)blockIdx.z * ell + j) * nchunk + blockIdx.x] = s;
            continue;
        }
        for (int t = lane * V; t < cnt; t += 32 * V) {
            TA u[V], zv[V];
            load_vec_pol<TU, TA, V>(uj + t, u, pol);
            lds_vec<TA, V>(zs + t, zv);
#pragma unroll
            for (int k = 0; k < V; ++k) s = fma(u[k], zv[k], s);
        }
        s = warp_sum(s);
        if (lane == 0) part[((size_t)blockIdx.z * ell + j) * nchunk + blockIdx.x] = s;
    }
}

template <class TU, class TZ, class TA>
int precond_vec(nys_ctx* ctx, const nys_precond* pc, int inverse, const void* z, void* out, int batch) {
    constexpr int V = Vec16<TU>::n;
    const nys_precond_priv* pv = (const nys_precond_priv*)pc->priv;
    const int64_t N = pc->N;
    const int ell = pv->ell_eff;   // only the columns with d > 0
    if (ell == 0) {
        if (out != z) NYS_CK(ctx, cudaMemcpyAsync(out, z, (size_t)batch * N * sizeof(TZ), cudaMemcpyDeviceToDevice,
                                                  ctx->stream));
        return NYS_OK;
    }
    const int nchunk = (int)((N + VCH - 1) / VCH);
    // column groups: about four CTAs per SM for the U^T z pass
    int groups = std::max(1, std::min(ell, (4 * ctx->sm_count + nchunk - 1) / nchunk));
    const int jper = (ell + groups - 1) / groups;
    groups = (ell + jper - 1) / jper;
    if (batch > 65535) return fail(ctx, NYS_EINVAL, "precond: batch above 65535");
    int st;
    TA* part = (TA*)scratch(ctx, SLOT_PRECOND, ((size_t)batch * nchunk * ell + 2 * (size_t)batch * ell) * sizeof(TA), &st);
    if (st) return st;
    TA* coef = part + (size_t)batch * nchunk * ell;
    TA* wbuf = coef + (size_t)batch * ell;
    cudaStream_t s = ctx->stream;
    const int keep = l2_keep_cols(ctx, N, sizeof(TU), ell);
    NYS_CK(ctx, launch_pdl(utz_vec_kernel<TU, TZ, TA>, dim3(nchunk, groups, batch), 256, 0, s, (const TU*)pc->U,
                           (const TZ*)z, N, ell, jper, part, keep));
    NYS_LAUNCH_CK(ctx);
    using TM = typename std::conditional<sizeof(TA) == 8, double, float>::type;
    const TM* Mp = sizeof(TA) == 8 ? (const TM*)pv->M64 : (const TM*)pv->M32;
    const TM* dp = sizeof(TA) == 8 ? (const TM*)pv->d : (const TM*)pv->d32;
    if ((st = coef_run<TA, TM>(ctx, part, nchunk, ell, pc->ell, inverse, Mp, dp, coef, batch, wbuf))) return st;
    // large active sets: two 16-byte vectors per lane and two columns per
    // round (1 KB contiguous per column and warp, near the HBM rate)
    const int pvx = ell <= 64 ? 1 : 2;
    const int P = 32 * V * pvx;
    const size_t sm = (((size_t)ell + 3) & ~size_t(3)) * sizeof(TA) + (size_t)8 * P * sizeof(TA);
    const dim3 grid((unsigned)((N + P - 1) / P), batch);
    if (pvx == 1)
        NYS_CK(ctx, launch_pdl(uc_vec_kernel<TU, TZ, TA>, grid, 256, sm, s, (const TU*)pc->U, (const TZ*)z, N, ell,
                               coef, inverse ? TA(-1) : TA(1), (TZ*)out, (const TZ*)nullptr, TA(1), keep,
                               DualStop{}));
    else
        NYS_CK(ctx, launch_pdl(uc_vec_kernel<TU, TZ, TA, 2, 2>, grid, 256, sm, s, (const TU*)pc->U, (const TZ*)z, N,
                               ell, coef, inverse ? TA(-1) : TA(1), (TZ*)out, (const TZ*)nullptr, TA(1), keep,
                               DualStop{}));
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

// The two halves of the apply for a factor whose U holds only this rank's
// rows of a pixel-sharded problem (the ranks sum w between them):
//   partial:  w[b][j] = sum over the local rows of U[j][i] z[b][i]  (j < ell_active)
//   finish:   out[b] = z[b] -/+ U coef(w[b])  (coef = M w or d .* w)
template <class TU, class TZ, class TA>
int precond_partial_typed(nys_ctx* ctx, const nys_precond* pc, const void* z, TA* w, int batch) {
    const nys_precond_priv* pv = (const nys_precond_priv*)pc->priv;
    const int64_t N = pc->N;
    const int ell = pv->ell_eff;
    if (ell == 0) return NYS_OK;
    const int nchunk = (int)((N + VCH - 1) / VCH);
    int groups = std::max(1, std::min(ell, (4 * ctx->sm_count + nchunk - 1) / nchunk));
    const int jper = (ell + groups - 1) / groups;
    groups = (ell + jper - 1) / jper;
    int st;
    TA* part = (TA*)scratch(ctx, SLOT_PRECOND, (size_t)batch * nchunk * ell * sizeof(TA), &st);
    if (st) return st;
    cudaStream_t s = ctx->stream;
    const int keep = l2_keep_cols(ctx, N, sizeof(TU), ell);
    NYS_CK(ctx, launch_pdl(utz_vec_kernel<TU, TZ, TA>, dim3(nchunk, groups, batch), 256, 0, s, (const TU*)pc->U,
                           (const TZ*)z, N, ell, jper, part, keep));
    NYS_LAUNCH_CK(ctx);
    NYS_CK(ctx, launch_pdl(reduce_cols_kernel<TA>, dim3((ell + 7) / 8, batch), 256, 0, s, part, nchunk, ell, w,
                           DualStop{}));
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

template <class TU, class TZ, class TA>
int precond_finish_typed(nys_ctx* ctx, const nys_precond* pc, int inverse, const TA* w, const void* z, void* out,
                         int batch) {
    constexpr int V = Vec16<TU>::n;
    const nys_precond_priv* pv = (const nys_precond_priv*)pc->priv;
    const int64_t N = pc->N;
    const int ell = pv->ell_eff;
    cudaStream_t s = ctx->stream;
    if (ell == 0) {
        if (out != z) NYS_CK(ctx, cudaMemcpyAsync(out, z, (size_t)batch * N * sizeof(TZ), cudaMemcpyDeviceToDevice, s));
        return NYS_OK;
    }
    int st;
    TA* coef = (TA*)scratch(ctx, SLOT_MISC, (size_t)batch * ell * sizeof(TA) + 64, &st);
    if (st) return st;
    using TM = typename std::conditional<sizeof(TA) == 8, double, float>::type;
    const TM* Mp = sizeof(TA) == 8 ? (const TM*)pv->M64 : (const TM*)pv->M32;
    const TM* dp = sizeof(TA) == 8 ? (const TM*)pv->d : (const TM*)pv->d32;
    NYS_CK(ctx, launch_pdl(mw_kernel<TA, TM>, dim3((ell + 7) / 8, batch), 256, ell * sizeof(TA), s, Mp, pc->ell, inverse,
                           dp, w, ell, coef, DualStop{}));
    NYS_LAUNCH_CK(ctx);
    const int keep = l2_keep_cols(ctx, N, sizeof(TU), ell);
    const int P = 32 * V * 2;
    const size_t sm = (((size_t)ell + 3) & ~size_t(3)) * sizeof(TA) + (size_t)8 * P * sizeof(TA);
    NYS_CK(ctx, launch_pdl(uc_vec_kernel<TU, TZ, TA, 2, 2>, dim3((unsigned)((N + P - 1) / P), batch), 256, sm, s,
                           (const TU*)pc->U, (const TZ*)z, N, ell, coef, inverse ? TA(-1) : TA(1), (TZ*)out,
                           (const TZ*)nullptr, TA(1), keep, DualStop{}));
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

template <class TU, class TZ, class TA>
int precond_typed(nys_ctx* ctx, const nys_precond* pc, int inverse, const void* z, void* out, int batch) {
    const nys_precond_priv* pv = (const nys_precond_priv*)pc->priv;
    const int64_t N = pc->N;
    const int ell = pc->ell;
    {
        constexpr int V = Vec16<TU>::n;
        const bool aligned = (((uintptr_t)pc->U | (uintptr_t)z | (uintptr_t)out) & 15) == 0;
        if (N % V == 0 && N % 4 == 0 && aligned && batch <= 65535)
            return precond_vec<TU, TZ, TA>(ctx, pc, inverse, z, out, batch);
    }
    const int nb = (int)((N + PCH - 1) / PCH);
    // chunks of at most 65535 images (grid.y) run one after another on the
    // stream and reuse the same scratch
    const size_t bmax = (size_t)std::min(batch, 65535);
    int st;
    TA* part = (TA*)scratch(ctx, SLOT_PRECOND, (bmax * nb * ell + bmax * ell) * sizeof(TA), &st);
    if (st) return st;
    TA* coef = part + bmax * nb * ell;
    cudaStream_t s = ctx->stream;
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int bb = std::min(65535, batch - b0);
        utz_kernel<TU, TZ, TA><<<dim3(nb, bb), 256, 0, s>>>((const TU*)pc->U, (const TZ*)z + (size_t)b0 * N, N, ell,
                                                             part);
        NYS_LAUNCH_CK(ctx);
        if (sizeof(TA) == 8)
            coef_kernel<TA, double><<<dim3((ell + 31) / 32, bb), 256, ell * sizeof(double), s>>>(
                part, nb, ell, ell, inverse, (const double*)pv->M64, (const double*)pv->d, coef);
        else
            coef_kernel<TA, float><<<dim3((ell + 31) / 32, bb), 256, ell * sizeof(double), s>>>(
                part, nb, ell, ell, inverse, (const float*)pv->M32, (const float*)pv->d32, coef);
        NYS_LAUNCH_CK(ctx);
        const int gx = (int)std::min<int64_t>((N + 255) / 256, 4096);
        uc_kernel<TU, TZ, TA><<<dim3(gx, bb), 256, ell * sizeof(TA), s>>>(
            (const TU*)pc->U, (const TZ*)z + (size_t)b0 * N, N, ell, coef, inverse ? TA(-1) : TA(1),
            (TZ*)out + (size_t)b0 * N);
        NYS_LAUNCH_CK(ctx);
    }
    return NYS_OK;
}

int precond_setup_impl(nys_ctx* ctx, nys_precond* pc, double mu, int sqrt_shift) {
    auto* pv = (nys_precond_priv*)pc->priv;
    const int ell = pc->ell;
    const double sref = sqrt_shift ? std::sqrt(std::max(pc->s_last, 0.0)) : pc->s_last;
    if (!(sref + mu > 0.0))
        return fail(ctx, NYS_EDEGENERATE, "preconditioner: s_K%s + mu = %g is not positive",
                    sqrt_shift ? " (square-rooted)" : "", sref + mu);
    cudaStream_t s = ctx->stream;
    // active prefix: the same IEEE double expression as weights_kernel; d is
    // non-increasing, so d_i > 0 exactly for i < eff
    std::vector<double> S(ell);
    NYS_CK(ctx, cudaMemcpyAsync(S.data(), pc->S_hat, ell * sizeof(double), cudaMemcpyDeviceToHost, s));
    NYS_CK(ctx, cudaStreamSynchronize(s));
    int eff = 0;
    for (int i = 0; i < ell; ++i)
        if ((S[i] + mu) / (sref + mu) - 1.0 > 0.0) eff = i + 1;
    int st;
    double* work = (double*)scratch(ctx, SLOT_FACTOR, (size_t)3 * ell * ell * sizeof(double) + 256, &st);
    if (st) return st;
    double* A = work;
    double* Li = A + (size_t)ell * ell;
    double* Ai = Li + (size_t)ell * ell;
    double* info = Ai + (size_t)ell * ell;
    NYS_CK(ctx, cudaMemsetAsync(info, 0, 4 * sizeof(double), s));
    weights_kernel<<<(ell + 127) / 128, 128, 0, s>>>(pc->S_hat, ell, mu, sqrt_shift, pv->d, pv->sqrtd, pv->d32);
    NYS_LAUNCH_CK(ctx);
    if (eff > 0) {
        // (I + Ubar^T Ubar)^{-1} on the active block only (Ubar's other columns are 0)
        form_A_kernel<<<64, 256, 0, s>>>(pv->K, ell, pv->sqrtd, eff, A);
        NYS_LAUNCH_CK(ctx);
        st = chol_cluster(ctx, A, eff, eff, 0, 0.0, 0, A, info, 3);
        if (st == NYS_EINVAL) {
            chol_kernel<<<1, 1024, 0, s>>>(A, eff, info);
            NYS_LAUNCH_CK(ctx);
        } else if (st) {
            return st;
        }
        tri_inv_kernel<<<eff, 32, eff * sizeof(double), s>>>(A, Li, eff);
        NYS_LAUNCH_CK(ctx);
        // (I + Ubar^T Ubar)^{-1} = L^{-T} L^{-1}
        if ((st = launch_small_gemm(ctx, Li, 1, Li, 0, eff, eff, eff, nullptr, Ai))) return st;
    }
    form_M_kernel<<<64, 256, 0, s>>>(Ai, pv->sqrtd, ell, eff, pv->M64, pv->M32);
    NYS_LAUNCH_CK(ctx);
    double h_info[4];
    NYS_CK(ctx, cudaMemcpyAsync(h_info, info, sizeof(h_info), cudaMemcpyDeviceToHost, s));
    NYS_CK(ctx, cudaStreamSynchronize(s));
    if (h_info[3] != 0.0) return fail(ctx, NYS_ENONFINITE, "preconditioner: I + Ubar^T Ubar is not positive definite");
    pv->ell_eff = eff;
    pc->ell_active = eff;
    pc->mu = mu;
    pc->sqrt_shift = sqrt_shift;
    return NYS_OK;
}

}  // namespace

int precond_run(nys_ctx* ctx, const nys_precond* pc, int inverse, int dtype, const void* z, void* out, int batch) {
    if (!pc || !pc->priv || !pc->U) return fail(ctx, NYS_EINVAL, "precond: not factored");
    if (pc->mu != pc->mu) return fail(ctx, NYS_EINVAL, "precond: call nys_precond_setup first");
    if (dtype == NYS_F64) {
        if (pc->dtype != NYS_F64) return fail(ctx, NYS_EINVAL, "precond: f64 data needs an f64 factor");
        return precond_typed<double, double, double>(ctx, pc, inverse, z, out, batch);
    }
    if (dtype != NYS_F32) return fail(ctx, NYS_EINVAL, "precond: data must be f32 or f64");
    if (pc->dtype == NYS_F32) return precond_typed<float, float, float>(ctx, pc, inverse, z, out, batch);
    if (pc->dtype == NYS_BF16) return precond_typed<__nv_bfloat16, float, float>(ctx, pc, inverse, z, out, batch);
    return fail(ctx, NYS_EINVAL, "precond: f32 data needs an f32 or bf16 factor");
}

// Omega (total entries of store_dt, starting at element `first` of the
// generator's stream) from the counter-based generator
int omega_fill(nys_ctx* ctx, int store_dt, void* Omega, int64_t total, uint64_t seed, int64_t first) {
    cudaStream_t s = ctx->stream;
    const int grid = (int)std::min<int64_t>((total / 4 + 255) / 256 + 1, ctx->sm_count * 16);
    if (store_dt == NYS_F64) omega_kernel<double, double><<<grid, 256, 0, s>>>((double*)Omega, first, total, seed);
    else if (store_dt == NYS_F32) omega_kernel<float, float><<<grid, 256, 0, s>>>((float*)Omega, first, total, seed);
    else omega_kernel<__nv_bfloat16, float><<<grid, 256, 0, s>>>((__nv_bfloat16*)Omega, first, total, seed);
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

}  // namespace nys

using namespace nys;

extern "C" {

int nys_sketch(nys_ctx* ctx, nys_op* op, int phi_kind, int ell, uint64_t seed, int store_dt, void* Omega, void* Y) {
    return nys_sketch_cols(ctx, op, phi_kind, ell, 0, ell, seed, store_dt, Omega, Y);
}

int nys_sketch_cols(nys_ctx* ctx, nys_op* op, int phi_kind, int ell_total, int j0, int j1, uint64_t seed,
                    int store_dt, void* Omega, void* Y) {
    if (!ctx || !op || !Omega || !Y) return fail(ctx, NYS_EINVAL, "nys_sketch: null argument");
    if (ell_total <= 0 || j0 < 0 || j1 <= j0 || j1 > ell_total)
        return fail(ctx, NYS_EINVAL, "nys_sketch: need 0 <= j0 < j1 <= ell");
    const int ell = j1 - j0;
    if (op->dtype == NYS_F64 ? store_dt != NYS_F64 : (store_dt != NYS_F32 && store_dt != NYS_BF16))
        return fail(ctx, NYS_EINVAL, "nys_sketch: store dtype does not match the operator");
    if (phi_kind == NYS_PHI_W_ATA_WT && op->haar_levels <= 0)
        return fail(ctx, NYS_EINVAL, "nys_sketch: W A^T A W^T needs an operator with haar_levels");
    if (int st0 = omega_fill(ctx, store_dt, Omega, (int64_t)ell * op->N, seed, (int64_t)j0 * op->N)) return st0;
    if (phi_kind == NYS_PHI_ATA) return op_run(op, 2, Omega, Y, ell, store_dt, store_dt);
    if (phi_kind != NYS_PHI_W_ATA_WT) return fail(ctx, NYS_EINVAL, "nys_sketch: unknown phi kind");
    // W A^T A W^T, chunked through compute-type temporaries
    const int cdt = op->dtype;
    const size_t es = dtype_size(cdt);
    const int chunk = std::min(ell, 64);
    int st;
    char* tmp = (char*)scratch(ctx, SLOT_SKETCH, 2 * (size_t)chunk * op->N * es, &st);
    if (st) return st;
    char* t1 = tmp;
    char* t2 = tmp + (size_t)chunk * op->N * es;
    const size_t ss = dtype_size(store_dt);
    for (int b0 = 0; b0 < ell; b0 += chunk) {
        const int nb = std::min(chunk, ell - b0);
        const char* om = (const char*)Omega + (size_t)b0 * op->N * ss;
        char* yy = (char*)Y + (size_t)b0 * op->N * ss;
        if ((st = haar_run(op, om, t1, nb, 1, store_dt, cdt))) return st;
        if ((st = op_run(op, 2, t1, t2, nb, cdt, cdt))) return st;
        if ((st = haar_run(op, t2, yy, nb, 0, cdt, store_dt))) return st;
    }
    return NYS_OK;
}

int nys_precond_release(nys_precond* pc) {
    if (!pc || !pc->priv) return NYS_OK;
    auto* pv = (nys_precond_priv*)pc->priv;
    cudaDeviceSynchronize();
    void* bufs[] = {pv->K, pv->d, pv->M64, pv->M32, pv->d32, pv->sqrtd};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete pv;
    pc->priv = nullptr;
    return NYS_OK;
}

// allocate (or re-size) the library-owned small state of a preconditioner
static int alloc_priv(nys_ctx* ctx, nys_precond* pc) {
    const int ell = pc->ell;
    if (pc->priv && ((nys_precond_priv*)pc->priv)->ell != ell) nys_precond_release(pc);
    if (pc->priv) return NYS_OK;
    auto* pv = new nys_precond_priv();
    pv->ell = ell;
    const size_t l2 = (size_t)ell * ell;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&pv->K, l2 * 8);
    if (e == cudaSuccess) e = cudaMalloc(&pv->M64, l2 * 8);
    if (e == cudaSuccess) e = cudaMalloc(&pv->M32, l2 * 4);
    if (e == cudaSuccess) e = cudaMalloc(&pv->d, ell * 8);
    if (e == cudaSuccess) e = cudaMalloc(&pv->sqrtd, ell * 8);
    if (e == cudaSuccess) e = cudaMalloc(&pv->d32, ell * 4);
    pc->priv = pv;
    if (e != cudaSuccess) {
        nys_precond_release(pc);
        return cuda_fail(ctx, e, "preconditioner state: cudaMalloc");
    }
    return NYS_OK;
}

// The ell x ell part of Algorithm 1 (steps 3-8) from the Gram G2 of
// [Omega | Y] (2 ell x 2 ell, ld 2 ell, device): shift, shifted Cholesky,
// G = C^{-1} Y_v^T Y_v C^{-T} = B^T B, its eigen-decomposition, S_hat, and
// W = C^{-T} V S^{-1} (ell x ell, row-major, device) so that U = (Y + v Omega) W.
// info (device, 16 doubles): [0] status (1: Cholesky failed after the
// retries), [1] v, [2] retries.  Workspace from SLOT_FACTOR after `skip`
// doubles (room the caller keeps for G2).
static int factor_small(nys_ctx* ctx, const double* G2, int ell, double eps, bool eig_f32, size_t skip,
                        double* S_hat, double** W_out, double** info_out) {
    const size_t l2 = (size_t)ell * ell;
    const int n = (ell + 1) & ~1;
    int st;
    // layout after the skipped doubles (float64 unless noted): C, H, Ci, T1,
    // Gm, Vs, scale, info (16) + sweeps (16), then the eigen work area: 2 n^2
    // values of the Jacobi type and ell doubles
    const size_t need = (skip + 6 * l2 + (size_t)ell + 32) * 8 + 2 * (size_t)n * n * 8 + 8 * (size_t)n + 256;
    double* w = (double*)scratch(ctx, SLOT_FACTOR, need, &st);
    if (st) return st;
    double* C = w + skip;
    double* H = C + l2;
    double* Ci = H + l2;
    double* T1 = Ci + l2;
    double* Gm = T1 + l2;
    double* Vs = Gm + l2;
    double* scale = Vs + l2;
    double* info = scale + ell;           // 16 doubles
    int* sweeps = (int*)(info + 16);
    void* ework = (void*)(info + 32);     // eigen work (2 n^2 T + n doubles)
    cudaStream_t s = ctx->stream;
    NYS_CK(ctx, cudaMemsetAsync(info, 0, 16 * sizeof(double), s));
    // shifted Cholesky (steps 4-5): on a 16-SM cluster where it fits, else one CTA
    st = chol_cluster(ctx, G2, 2 * ell, ell, 1, eps, 8, C, info, 0);
    if (st == NYS_EINVAL) {
        shift_chol_kernel<<<1, 1024, 0, s>>>(G2, ell, eps, 8, C, info);
        NYS_LAUNCH_CK(ctx);
    } else if (st) {
        return st;
    }
    form_H_kernel<<<64, 256, 0, s>>>(G2, ell, info, H);
    NYS_LAUNCH_CK(ctx);
    tri_inv_kernel<<<ell, 32, ell * sizeof(double), s>>>(C, Ci, ell);
    NYS_LAUNCH_CK(ctx);
    if ((st = launch_small_gemm(ctx, Ci, 0, H, 0, ell, ell, ell, nullptr, T1))) return st;
    if ((st = launch_small_gemm(ctx, T1, 0, Ci, 1, ell, ell, ell, nullptr, Gm))) return st;
    if ((st = sym_eig(ctx, Gm, ell, eig_f32, info, ework, Vs, S_hat, scale, sweeps))) return st;
    // W = C^{-T} V S^{-1}  (into T1)
    if ((st = launch_small_gemm(ctx, Ci, 1, Vs, 0, ell, ell, ell, scale, T1))) return st;
    *W_out = T1;
    *info_out = info;
    return NYS_OK;
}

int nys_factor(nys_ctx* ctx, const void* Omega, const void* Y, int in_dt, int64_t N, int ell, double eps,
               nys_precond* pc) {
    if (!ctx || !Omega || !Y || !pc || !pc->U || !pc->S_hat) return fail(ctx, NYS_EINVAL, "nys_factor: null argument");
    if (N <= 0 || ell <= 0 || ell > 1024 || ell > N)
        return fail(ctx, NYS_EINVAL, "nys_factor: need 0 < ell <= min(N, 1024)");
    if (!(eps >= 0.0)) return fail(ctx, NYS_EINVAL, "nys_factor: eps must be >= 0");
    const bool f64 = in_dt == NYS_F64;
    if (f64 != (pc->dtype == NYS_F64)) return fail(ctx, NYS_EINVAL, "nys_factor: f64 data needs an f64 factor");
    if (!f64 && in_dt != NYS_F32 && in_dt != NYS_BF16) return fail(ctx, NYS_EINVAL, "nys_factor: bad input dtype");
    pc->N = N;
    pc->ell = ell;
    if (int st0 = alloc_priv(ctx, pc)) return st0;
    auto* pv = (nys_precond_priv*)pc->priv;
    pc->mu = NAN;
    const int L2 = 2 * ell;
    const size_t l2 = (size_t)ell * ell;
    const int n = (ell + 1) & ~1;
    int st;
    // G2 at the start of the factor workspace, sized for factor_small too
    const size_t need = ((size_t)L2 * L2 + 6 * l2 + (size_t)ell + 32) * 8 + 2 * (size_t)n * n * 8 + 8 * (size_t)n + 256;
    double* G2 = (double*)scratch(ctx, SLOT_FACTOR, need, &st);
    if (st) return st;
    cudaStream_t s = ctx->stream;
    // one Gram pass over [Omega | Y]: Omega^T Omega, Omega^T Y and Y^T Y in
    // one tensor-core launch for bf16 sketches, three passes otherwise
    st = NYS_EINVAL;
    if (in_dt == NYS_BF16) {
        const void* srcs[2] = {Omega, Y};
        const int cols[2] = {ell, ell};
        const GramJob jobs[3] = {{0, 0, G2, L2}, {0, 1, G2 + ell, L2}, {1, 1, G2 + (size_t)ell * L2 + ell, L2}};
        st = gram_tc_jobs(ctx, srcs, cols, 2, N, 3, jobs);
        if (st != NYS_OK && st != NYS_EINVAL) return st;
    }
    if (st == NYS_EINVAL) {
        if ((st = gram_AtB(ctx, in_dt, Omega, ell, Omega, ell, N, G2, L2))) return st;
        if ((st = gram_AtB(ctx, in_dt, Omega, ell, Y, ell, N, G2 + ell, L2))) return st;
        if ((st = gram_AtB(ctx, in_dt, Y, ell, Y, ell, N, G2 + (size_t)ell * L2 + ell, L2))) return st;
    }
    double* T1 = nullptr;
    double* info = nullptr;
    if ((st = factor_small(ctx, G2, ell, eps, !f64, (size_t)L2 * L2, pc->S_hat, &T1, &info))) return st;
    // U = (Y + v Omega) W
    if ((st = gemm_tall(ctx, in_dt, Y, Omega, info + 1, N, ell, T1, ell, pc->dtype, pc->U))) return st;
    // K = U^T U of the stored U
    if ((st = gram_AtB(ctx, pc->dtype, pc->U, ell, pc->U, ell, N, pv->K, ell))) return st;
    double h[4];
    NYS_CK(ctx, cudaMemcpyAsync(h, info, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    NYS_CK(ctx, cudaMemcpyAsync(&pc->s_first, pc->S_hat, sizeof(double), cudaMemcpyDeviceToHost, s));
    NYS_CK(ctx, cudaMemcpyAsync(&pc->s_last, pc->S_hat + ell - 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    NYS_CK(ctx, cudaStreamSynchronize(s));
    if (int st2 = check_tc_timeout(ctx)) return st2;
    pc->v = h[1];
    pc->chol_retries = (int)h[2];
    if (h[0] != 0.0) return fail(ctx, NYS_ENOTSPD, "nys_factor: Cholesky of the shifted core failed after %d retries",
                                 pc->chol_retries);
    if (!std::isfinite(pc->s_first) || !std::isfinite(pc->s_last))
        return fail(ctx, NYS_ENONFINITE, "nys_factor: non-finite eigenvalues");
    // default preconditioner set-up (skipped when s_K is zero: set mu > 0 then)
    const double sref = std::sqrt(std::max(pc->s_last, 0.0));
    if (sref > 0.0) return precond_setup_impl(ctx, pc, 0.0, 1);
    return NYS_OK;
}

int nys_precond_import(nys_ctx* ctx, nys_precond* pc, double mu, int sqrt_shift) {
    if (!ctx || !pc || !pc->U || !pc->S_hat) return fail(ctx, NYS_EINVAL, "nys_precond_import: null argument");
    const int ell = pc->ell;
    if (pc->N <= 0 || ell <= 0 || ell > 1024 || ell > pc->N)
        return fail(ctx, NYS_EINVAL, "nys_precond_import: need 0 < ell <= min(N, 1024)");
    if (pc->dtype != NYS_F32 && pc->dtype != NYS_F64 && pc->dtype != NYS_BF16)
        return fail(ctx, NYS_EINVAL, "nys_precond_import: bad dtype");
    if (int st = alloc_priv(ctx, pc)) return st;
    auto* pv = (nys_precond_priv*)pc->priv;
    pc->mu = NAN;
    int st;
    if ((st = gram_AtB(ctx, pc->dtype, pc->U, ell, pc->U, ell, pc->N, pv->K, ell))) return st;
    cudaStream_t s = ctx->stream;
    NYS_CK(ctx, cudaMemcpyAsync(&pc->s_first, pc->S_hat, sizeof(double), cudaMemcpyDeviceToHost, s));
    NYS_CK(ctx, cudaMemcpyAsync(&pc->s_last, pc->S_hat + ell - 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    NYS_CK(ctx, cudaStreamSynchronize(s));
    return precond_setup_impl(ctx, pc, mu, sqrt_shift ? 1 : 0);
}

int nys_factor_gram(nys_ctx* ctx, const double* G2, int ell, double eps, int eig_f64, double* W, double* S_hat,
                    double* v, int* retries) {
    if (!ctx || !G2 || !W || !S_hat) return fail(ctx, NYS_EINVAL, "nys_factor_gram: null argument");
    if (ell <= 0 || ell > 1024) return fail(ctx, NYS_EINVAL, "nys_factor_gram: need 0 < ell <= 1024");
    if (!(eps >= 0.0)) return fail(ctx, NYS_EINVAL, "nys_factor_gram: eps must be >= 0");
    int st;
    double* T1 = nullptr;
    double* info = nullptr;
    if ((st = factor_small(ctx, G2, ell, eps, eig_f64 == 0, 0, S_hat, &T1, &info))) return st;
    cudaStream_t s = ctx->stream;
    NYS_CK(ctx, cudaMemcpyAsync(W, T1, (size_t)ell * ell * sizeof(double), cudaMemcpyDeviceToDevice, s));
    double h[3];
    NYS_CK(ctx, cudaMemcpyAsync(h, info, sizeof(h), cudaMemcpyDeviceToHost, s));
    NYS_CK(ctx, cudaStreamSynchronize(s));
    if (v) *v = h[1];
    if (retries) *retries = (int)h[2];
    if (h[0] != 0.0) return fail(ctx, NYS_ENOTSPD, "nys_factor_gram: Cholesky of the shifted core failed after %d "
                                 "retries", (int)h[2]);
    return NYS_OK;
}

int nys_precond_import_gram(nys_ctx* ctx, nys_precond* pc, const double* K, double mu, int sqrt_shift) {
    if (!ctx || !pc || !pc->U || !pc->S_hat || !K) return fail(ctx, NYS_EINVAL, "nys_precond_import_gram: null argument");
    const int ell = pc->ell;
    if (pc->N <= 0 || ell <= 0 || ell > 1024)
        return fail(ctx, NYS_EINVAL, "nys_precond_import_gram: need N > 0 and 0 < ell <= 1024");
    if (pc->dtype != NYS_F32 && pc->dtype != NYS_F64 && pc->dtype != NYS_BF16)
        return fail(ctx, NYS_EINVAL, "nys_precond_import_gram: bad dtype");
    if (int st = alloc_priv(ctx, pc)) return st;
    auto* pv = (nys_precond_priv*)pc->priv;
    pc->mu = NAN;
    cudaStream_t s = ctx->stream;
    NYS_CK(ctx, cudaMemcpyAsync(pv->K, K, (size_t)ell * ell * sizeof(double), cudaMemcpyDeviceToDevice, s));
    NYS_CK(ctx, cudaMemcpyAsync(&pc->s_first, pc->S_hat, sizeof(double), cudaMemcpyDeviceToHost, s));
    NYS_CK(ctx, cudaMemcpyAsync(&pc->s_last, pc->S_hat + ell - 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    NYS_CK(ctx, cudaStreamSynchronize(s));
    return precond_setup_impl(ctx, pc, mu, sqrt_shift ? 1 : 0);
}

int nys_precond_setup(nys_ctx* ctx, nys_precond* pc, double mu, int sqrt_shift) {
    if (!ctx || !pc || !pc->priv) return fail(ctx, NYS_EINVAL, "nys_precond_setup: factor first");
    return precond_setup_impl(ctx, pc, mu, sqrt_shift ? 1 : 0);
}

// shared checks of the split apply: vector path only (N a multiple of the
// 16-byte vector width, aligned operands), batch <= 65535
static int split_check(nys_ctx* ctx, const nys_precond* pc, int dtype, const void* a, const void* b, int batch,
                       const char* who) {
    if (!ctx || !pc || !a || !b) return fail(ctx, NYS_EINVAL, "%s: null argument", who);
    if (!pc->priv || !pc->U || pc->mu != pc->mu) return fail(ctx, NYS_EINVAL, "%s: preconditioner not set up", who);
    if (batch < 1 || batch > 65535) return fail(ctx, NYS_EINVAL, "%s: batch must be in [1, 65535]", who);
    const int V = pc->dtype == NYS_BF16 ? 8 : (pc->dtype == NYS_F32 ? 4 : 2);
    if (pc->N % V || pc->N % 4 || (((uintptr_t)pc->U | (uintptr_t)a | (uintptr_t)b) & 15))
        return fail(ctx, NYS_EINVAL, "%s: rows must be a multiple of %d and buffers 16-byte aligned", who, V);
    if (dtype == NYS_F64 ? pc->dtype != NYS_F64 : (dtype != NYS_F32 || pc->dtype == NYS_F64))
        return fail(ctx, NYS_EINVAL, "%s: data and factor dtypes do not match", who);
    return NYS_OK;
}

int precond_partial(nys_ctx* ctx, const nys_precond* pc, int dtype, const void* z, void* w, int batch) {
    if (int st = split_check(ctx, pc, dtype, z, w, batch, "precond_partial")) return st;
    if (dtype == NYS_F64) return precond_partial_typed<double, double, double>(ctx, pc, z, (double*)w, batch);
    if (pc->dtype == NYS_F32) return precond_partial_typed<float, float, float>(ctx, pc, z, (float*)w, batch);
    return precond_partial_typed<__nv_bfloat16, float, float>(ctx, pc, z, (float*)w, batch);
}

int precond_finish(nys_ctx* ctx, const nys_precond* pc, int inverse, int dtype, const void* w, const void* z,
                   void* out, int batch) {
    if (int st = split_check(ctx, pc, dtype, z, out, batch, "precond_finish")) return st;
    if (!w) return fail(ctx, NYS_EINVAL, "precond_finish: null argument");
    if (dtype == NYS_F64)
        return precond_finish_typed<double, double, double>(ctx, pc, inverse, (const double*)w, z, out, batch);
    if (pc->dtype == NYS_F32)
        return precond_finish_typed<float, float, float>(ctx, pc, inverse, (const float*)w, z, out, batch);
    return precond_finish_typed<__nv_bfloat16, float, float>(ctx, pc, inverse, (const float*)w, z, out, batch);
}

int precond_apply(nys_ctx* ctx, const nys_precond* pc, int inverse, int dtype, const void* z, void* out, int batch) {
    if (!ctx || !pc || !z || !out) return fail(ctx, NYS_EINVAL, "precond_apply: null argument");
    if (batch < 0) return fail(ctx, NYS_EINVAL, "precond_apply: negative batch");
    if (batch == 0) return NYS_OK;
    return precond_run(ctx, pc, inverse, dtype, z, out, batch);
}

}  // extern "C"

// ------------------------------------------- allocation-free P / P^{-1} ----
// precond_apply_noalloc computes what precond_apply computes, with the plain
// (unvectorised) kernels of precond_apply's general path -- per-block partial
// sums of U^T z, the coefficient pass, then z + U c -- over the active columns
// only (those with d_i > 0; M and d vanish outside them), one image at a
// time.  Its scratch (the partial sums and the coefficients) lives in one
// file-scope device array instead of the context workspace, so the call
// never allocates: for callers that must not call cudaMalloc (a stream that
// is being captured into a CUDA graph by someone else, a real-time loop with
// a fixed memory budget, a host that hands the library only its own
// buffers).  Every process that loads the library keeps this array on each
// GPU it uses until it exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NYS_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {nullptr};   // device address of the array, per device

// Device address of g_noalloc_scratch on ctx's device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress once per device, with that device current.
int noalloc_scratch(nys_ctx* ctx, void** out) {
    if (ctx->device < 0 || ctx->device >= 256) return fail(ctx, NYS_EINVAL, "precond_apply_noalloc: device id");
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[ctx->device]) {
        int cur = 0;
        NYS_CK(ctx, cudaGetDevice(&cur));
        NYS_CK(ctx, cudaSetDevice(ctx->device));
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        cudaSetDevice(cur);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_addr[ctx->device] = p;
    }
    *out = g_noalloc_addr[ctx->device];
    return NYS_OK;
}

template <class TU, class TZ, class TA>
int precond_noalloc_typed(nys_ctx* ctx, const nys_precond* pc, int inverse, const void* z, void* out, int batch,
                          void* scratch_dev) {
    const nys_precond_priv* pv = (const nys_precond_priv*)pc->priv;
    const int64_t N = pc->N;
    const int ell = pv->ell_eff;   // active columns; M's leading dimension stays pc->ell
    const int ldm = pc->ell;
    const int nb = (int)((N + PCH - 1) / PCH);
    const size_t need = ((size_t)nb * ell + (size_t)ell) * sizeof(TA);
    if (need > NYS_NOALLOC_SCRATCH_BYTES)
        return fail(ctx, NYS_EINVAL,
                    "precond_apply_noalloc: needs %zu scratch bytes (ceil(N/%d) * ell_active + ell_active values) "
                    "but the fixed array holds %d; use precond_apply", need, PCH, (int)NYS_NOALLOC_SCRATCH_BYTES);
    if (ell == 0) {   // P = I: a device-to-device copy (no allocation)
        if (out != z) NYS_CK(ctx, cudaMemcpyAsync(out, z, (size_t)batch * N * sizeof(TZ), cudaMemcpyDeviceToDevice,
                                                  ctx->stream));
        return NYS_OK;
    }
    // every partial and coefficient is written before it is read: nothing
    // has to be cleared between calls
    TA* part = (TA*)scratch_dev;
    TA* coef = part + (size_t)nb * ell;
    cudaStream_t s = ctx->stream;
    const int gx = (int)std::min<int64_t>((N + 255) / 256, 4096);
    for (int b = 0; b < batch; ++b) {
        const TZ* zb = (const TZ*)z + (size_t)b * N;
        TZ* ob = (TZ*)out + (size_t)b * N;
        utz_kernel<TU, TZ, TA><<<dim3(nb, 1), 256, 0, s>>>((const TU*)pc->U, zb, N, ell, part);
        NYS_LAUNCH_CK(ctx);
        if (sizeof(TA) == 8)
            coef_kernel<TA, double><<<dim3((ell + 31) / 32, 1), 256, ell * sizeof(double), s>>>(
                part, nb, ell, ldm, inverse, (const double*)pv->M64, (const double*)pv->d, coef);
        else
            coef_kernel<TA, float><<<dim3((ell + 31) / 32, 1), 256, ell * sizeof(double), s>>>(
                part, nb, ell, ldm, inverse, (const float*)pv->M32, (const float*)pv->d32, coef);
        NYS_LAUNCH_CK(ctx);
        uc_kernel<TU, TZ, TA><<<dim3(gx, 1), 256, ell * sizeof(TA), s>>>((const TU*)pc->U, zb, N, ell, coef,
                                                                        inverse ? TA(-1) : TA(1), ob);
        NYS_LAUNCH_CK(ctx);
    }
    return NYS_OK;
}
}  // namespace

extern "C" int precond_apply_noalloc(nys_ctx* ctx, const nys_precond* pc, int inverse, int dtype, const void* z,
                                     void* out, int batch) {
    if (!ctx || !pc || !z || !out) return fail(ctx, NYS_EINVAL, "precond_apply_noalloc: null argument");
    if (batch < 0) return fail(ctx, NYS_EINVAL, "precond_apply_noalloc: negative batch");
    if (!pc->priv || !pc->U) return fail(ctx, NYS_EINVAL, "precond_apply_noalloc: not factored");
    if (pc->mu != pc->mu) return fail(ctx, NYS_EINVAL, "precond_apply_noalloc: call nys_precond_setup first");
    if (batch == 0) return NYS_OK;
    void* sp = nullptr;
    if (int st = noalloc_scratch(ctx, &sp)) return st;
    if (dtype == NYS_F64) {
        if (pc->dtype != NYS_F64) return fail(ctx, NYS_EINVAL, "precond_apply_noalloc: f64 data needs an f64 factor");
        return precond_noalloc_typed<double, double, double>(ctx, pc, inverse, z, out, batch, sp);
    }
    if (dtype != NYS_F32) return fail(ctx, NYS_EINVAL, "precond_apply_noalloc: data must be f32 or f64");
    if (pc->dtype == NYS_F32) return precond_noalloc_typed<float, float, float>(ctx, pc, inverse, z, out, batch, sp);
    if (pc->dtype == NYS_BF16)
        return precond_noalloc_typed<__nv_bfloat16, float, float>(ctx, pc, inverse, z, out, batch, sp);
    return fail(ctx, NYS_EINVAL, "precond_apply_noalloc: f32 data needs an f32 or bf16 factor");
}
