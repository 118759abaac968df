// Dense linear algebra of Algorithm 1 steps 3-8 on CUDA cores.
//
//  * gram_AtB   C = A^T B for tall N x p and N x q operands stored column by
//               column (each column an image).  Split-K over N: every CTA
//               accumulates a 64 x 64 output tile over one K range with 4 x 4
//               register micro-tiles; partial tiles are summed in float64 by a
//               second, deterministic pass (no atomics).
//  * gemm_tall  out = (A + alpha A2) W with A, A2: N x k, W: k x q (float64,
//               converted to the compute type), out: N x q.  128 x 64 output
//               tiles, 8 x 4 micro-tiles; the Y + v Omega of Algorithm 1 step 4
//               is formed while the A tile is loaded, so Y_v never exists in
//               memory.
//  * small ell x ell float64 kernels: shifted Cholesky with retries (one CTA),
//               triangular inverse (one warp per column), small GEMM, and the
//               cyclic parallel-order Jacobi eigensolver (one CTA).
#include "internal.cuh"

#include <cmath>

namespace nys {
namespace {

// ------------------------------------------------------------- gram ------
constexpr int GT = 64;   // output tile
constexpr int GK = 16;   // K step

template <class TI, class TA>
__global__ void __launch_bounds__(256) gram_kernel(const TI* __restrict__ A, int p, const TI* __restrict__ B, int q,
                                                   int64_t N, int64_t kchunk, TA* __restrict__ part) {
    __shared__ TA As[GK][GT + 4];
    __shared__ TA Bs[GK][GT + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int pi0 = blockIdx.y * GT, qj0 = blockIdx.x * GT;
    const int64_t k0 = blockIdx.z * kchunk;
    const int64_t k1 = min(N, k0 + kchunk);
    TA acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = TA(0);
    // loader: 256 threads load 64 columns x 16 k: thread -> (col = t / 4, k4 = (t % 4) * 4)
    const int lc = threadIdx.x >> 2, lk = (threadIdx.x & 3) * 4;
    for (int64_t kk = k0; kk < k1; kk += GK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t k = kk + lk + r;
            const int ca = pi0 + lc, cb = qj0 + lc;
            As[lk + r][lc] = (k < k1 && ca < p) ? (TA)ldf(A + (size_t)ca * N + k) : TA(0);
            Bs[lk + r][lc] = (k < k1 && cb < q) ? (TA)ldf(B + (size_t)cb * N + k) : TA(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GK; ++k) {
            TA av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[k][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
    TA* out = part + (size_t)blockIdx.z * p * q;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = pi0 + ty * 4 + a, j = qj0 + tx * 4 + b;
            if (i < p && j < q) out[(size_t)i * q + j] = acc[a][b];
        }
}

template <class TA>
__global__ void gram_reduce_kernel(const TA* __restrict__ part, int splits, int p, int q, double* __restrict__ C,
                                   int ldc) {
    const int64_t total = (int64_t)p * q;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < splits; ++z) s += (double)part[(size_t)z * total + t];
        const int i = (int)(t / q), j = (int)(t - (int64_t)i * q);
        C[(size_t)i * ldc + j] = s;
    }
}

// ------------------------------------------------------------- tall gemm -
constexpr int TM = 128, TN = 64, TK = 16;

template <class TI, class TO, class TA>
__global__ void __launch_bounds__(256) gemm_tall_kernel(const TI* __restrict__ A, const TI* __restrict__ A2,
                                                        const double* __restrict__ alpha_dev, int64_t N, int k, const TA* __restrict__ W, int q,
                                                        TO* __restrict__ out) {
    __shared__ TA As[TK][TM + 4];
    __shared__ TA Ws[TK][TN + 4];
    const int tx = threadIdx.x & 15;   // pixel group (8 pixels)
    const int ty = threadIdx.x >> 4;   // output group (4 outputs)
    const int64_t i0 = (int64_t)blockIdx.x * TM;
    const int j0 = blockIdx.y * TN;
    const TA alpha = alpha_dev ? (TA)*alpha_dev : TA(0);
    TA acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = TA(0);
    for (int kk = 0; kk < k; kk += TK) {
        // A tile: 16 k x 128 pixels; thread loads 8 pixels of one k
        {
            const int kr = threadIdx.x >> 4, pc = (threadIdx.x & 15) * 8;
            const int kc = kk + kr;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int64_t i = i0 + pc + r;
                TA v = TA(0);
                if (kc < k && i < N) {
                    v = (TA)ldf(A + (size_t)kc * N + i);
                    if (A2) v = fma(alpha, (TA)ldf(A2 + (size_t)kc * N + i), v);
                }
                As[kr][pc + r] = v;
            }
        }
        // W tile: 16 k x 64 outputs
        for (int t = threadIdx.x; t < TK * TN; t += 256) {
            const int kr = t / TN, jc = t - kr * TN;
            const int kc = kk + kr, j = j0 + jc;
            Ws[kr][jc] = (kc < k && j < q) ? W[(size_t)kc * q + j] : TA(0);
        }
        __syncthreads();
#pragma unroll
        for (int kr = 0; kr < TK; ++kr) {
            TA av[8], wv[4];
#pragma unroll
            for (int a = 0; a < 8; ++a) av[a] = As[kr][tx * 8 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) wv[b] = Ws[kr][ty * 4 + b];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], wv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int j = j0 + ty * 4 + b;
        if (j >= q) continue;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int64_t i = i0 + tx * 8 + a;
            if (i < N) stf(out + (size_t)j * N + i, acc[a][b]);
        }
    }
}

template <class TA>
__global__ void cast_kernel(const double* __restrict__ in, TA* __restrict__ out, int n) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) out[t] = (TA)in[t];
}

// ------------------------------------------------------------- norms -----
template <class T>
__global__ void norm2_diff_kernel(const T* __restrict__ a, const T* __restrict__ b, int64_t n, double* __restrict__ part) {
    __shared__ double sh[32];
    double s0 = 0.0, s1 = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const double av = (double)a[t];
        if (b) {
            const double bv = (double)b[t];
            s0 += (av - bv) * (av - bv);
            s1 += bv * bv;
        } else {
            s0 += av * av;
        }
    }
    s0 = block_sum(s0, sh);
    s1 = block_sum(s1, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s0;
        part[2 * blockIdx.x + 1] = s1;
    }
}

__global__ void sum_pairs_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
    __shared__ double sh[32];
    double s0 = 0.0, s1 = 0.0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) s0 += part[2 * t], s1 += part[2 * t + 1];
    s0 = block_sum(s0, sh);
    s1 = block_sum(s1, sh);
    if (threadIdx.x == 0) out[0] = s0, out[1] = s1;
}

}  // namespace

void gram_reduce_f32(nys_ctx* ctx, const float* part, int splits, int p, int q, double* C, int ldc, int blocks) {
    gram_reduce_kernel<float><<<blocks, 256, 0, ctx->stream>>>(part, splits, p, q, C, ldc);
}

int check_tc_timeout(nys_ctx* ctx) {
    if (ctx->slot_bytes[SLOT_TCERR] == 0) return NYS_OK;
    int h = 0;
    NYS_CK(ctx, cudaMemcpyAsync(&h, ctx->slot_ptr[SLOT_TCERR], sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    NYS_CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (h) return fail(ctx, NYS_ETIMEOUT, "a tensor-core kernel gave up waiting on its pipeline (bounded wait)");
    return NYS_OK;
}

int gram_AtB(nys_ctx* ctx, int dtype, const void* A, int p, const void* B, int q, int64_t N, double* C, int ldc) {
    return gram_AtB_path(ctx, dtype, A, p, B, q, N, C, ldc, 0);
}

int gram_AtB_path(nys_ctx* ctx, int dtype, const void* A, int p, const void* B, int q, int64_t N, double* C, int ldc,
                  int path) {
    if (N <= 0 || p <= 0 || q <= 0) return fail(ctx, NYS_EINVAL, "gram_AtB: empty operand");
    if (path != 1 && dtype == NYS_BF16) {
        const int st = gram_AtB_tc(ctx, A, p, B, q, N, C, ldc);
        if (st != NYS_EINVAL) return st;
        if (path == 2) return fail(ctx, NYS_EINVAL, "gram: shape not supported by the tensor-core path");
    } else if (path == 2) {
        return fail(ctx, NYS_EINVAL, "gram: the tensor-core path takes bf16 operands");
    }
    const int tiles = ((p + GT - 1) / GT) * ((q + GT - 1) / GT);
    // enough CTAs to fill the GPU about twice, each K range a multiple of GK
    int64_t splits = std::max<int64_t>(1, (2LL * ctx->sm_count + tiles - 1) / tiles);
    int64_t kchunk = (N + splits - 1) / splits;
    kchunk = std::max<int64_t>(GK, (kchunk + GK - 1) / GK * GK);
    splits = (N + kchunk - 1) / kchunk;
    const bool f64 = dtype == NYS_F64;
    const size_t ab = f64 ? 8 : 4;
    int st;
    void* part = scratch(ctx, SLOT_GRAM, (size_t)splits * p * q * ab, &st);
    if (st) return st;
    dim3 grid((q + GT - 1) / GT, (p + GT - 1) / GT, (unsigned)splits);
    if (f64)
        gram_kernel<double, double><<<grid, 256, 0, ctx->stream>>>((const double*)A, p, (const double*)B, q, N, kchunk,
                                                                  (double*)part);
    else if (dtype == NYS_F32)
        gram_kernel<float, float><<<grid, 256, 0, ctx->stream>>>((const float*)A, p, (const float*)B, q, N, kchunk,
                                                                (float*)part);
    else
        gram_kernel<__nv_bfloat16, float><<<grid, 256, 0, ctx->stream>>>(
            (const __nv_bfloat16*)A, p, (const __nv_bfloat16*)B, q, N, kchunk, (float*)part);
    NYS_LAUNCH_CK(ctx);
    const int rb = std::min<int64_t>(1024, ((int64_t)p * q + 255) / 256);
    if (f64)
        gram_reduce_kernel<double><<<rb, 256, 0, ctx->stream>>>((const double*)part, (int)splits, p, q, C, ldc);
    else
        gram_reduce_kernel<float><<<rb, 256, 0, ctx->stream>>>((const float*)part, (int)splits, p, q, C, ldc);
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

int gemm_tall(nys_ctx* ctx, int in_dt, const void* A, const void* A2, const double* alpha, int64_t N, int k,
              const double* W, int q, int out_dt, void* out) {
    return gemm_tall_path(ctx, in_dt, A, A2, alpha, N, k, W, q, out_dt, out, 0);
}

int gemm_tall_path(nys_ctx* ctx, int in_dt, const void* A, const void* A2, const double* alpha, int64_t N, int k,
                   const double* W, int q, int out_dt, void* out, int path) {
    if (path != 1 && in_dt == NYS_BF16 && A2 && k == q) {
        const int st = gemm_tall_tc(ctx, A, A2, alpha, N, k, W, out_dt, out);
        if (st != NYS_EINVAL) return st;
    }
    if (path == 2) return fail(ctx, NYS_EINVAL, "tall gemm: shape or dtype not supported by the tensor-core path");
    int st;
    const bool f64 = in_dt == NYS_F64;
    void* Wc = scratch(ctx, SLOT_MISC, (size_t)k * q * (f64 ? 8 : 4), &st);
    if (st) return st;
    dim3 grid((unsigned)((N + TM - 1) / TM), (q + TN - 1) / TN);
    if (f64) {
        if (out_dt != NYS_F64) return fail(ctx, NYS_EINVAL, "gemm_tall: f64 in needs f64 out");
        gemm_tall_kernel<double, double, double><<<grid, 256, 0, ctx->stream>>>(
            (const double*)A, (const double*)A2, alpha, N, k, W, q, (double*)out);
        NYS_LAUNCH_CK(ctx);
        return NYS_OK;
    }
    cast_kernel<float><<<64, 256, 0, ctx->stream>>>(W, (float*)Wc, k * q);
    NYS_LAUNCH_CK(ctx);
    const float* Wf = (const float*)Wc;
    const double* al = alpha;
    if (in_dt == NYS_F32 && out_dt == NYS_F32)
        gemm_tall_kernel<float, float, float><<<grid, 256, 0, ctx->stream>>>((const float*)A, (const float*)A2, al, N, k,
                                                                            Wf, q, (float*)out);
    else if (in_dt == NYS_BF16 && out_dt == NYS_BF16)
        gemm_tall_kernel<__nv_bfloat16, __nv_bfloat16, float><<<grid, 256, 0, ctx->stream>>>(
            (const __nv_bfloat16*)A, (const __nv_bfloat16*)A2, al, N, k, Wf, q, (__nv_bfloat16*)out);
    else if (in_dt == NYS_BF16 && out_dt == NYS_F32)
        gemm_tall_kernel<__nv_bfloat16, float, float><<<grid, 256, 0, ctx->stream>>>(
            (const __nv_bfloat16*)A, (const __nv_bfloat16*)A2, al, N, k, Wf, q, (float*)out);
    else if (in_dt == NYS_F32 && out_dt == NYS_BF16)
        gemm_tall_kernel<float, __nv_bfloat16, float><<<grid, 256, 0, ctx->stream>>>(
            (const float*)A, (const float*)A2, al, N, k, Wf, q, (__nv_bfloat16*)out);
    else
        return fail(ctx, NYS_EINVAL, "gemm_tall: unsupported dtypes");
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

int norm2_diff(nys_ctx* ctx, int dtype, int64_t n, const void* a, const void* b, double** out) {
    int st;
    const int nb = std::max(1, std::min<int>(ctx->sm_count * 4, (int)((n + 255) / 256)));
    double* buf = (double*)scratch(ctx, SLOT_MISC, (size_t)(nb + 1) * 2 * sizeof(double), &st);
    if (st) return st;
    double* out_dev = buf;
    double* part = buf + 2;
    *out = out_dev;
    if (dtype == NYS_F64)
        norm2_diff_kernel<double><<<nb, 256, 0, ctx->stream>>>((const double*)a, (const double*)b, n, part);
    else
        norm2_diff_kernel<float><<<nb, 256, 0, ctx->stream>>>((const float*)a, (const float*)b, n, part);
    NYS_LAUNCH_CK(ctx);
    sum_pairs_kernel<<<1, 256, 0, ctx->stream>>>(part, nb, out_dev);
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

}  // namespace nys
