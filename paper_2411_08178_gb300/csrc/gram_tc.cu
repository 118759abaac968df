// Tall-skinny Gram products C = A^T B on the 5th-generation tensor cores
// (tcgen05), several of them in one launch.
//
// The operands (at most two: Omega and Y, or U) hold their columns as
// contiguous bf16 images, so as MMA operands both sides are K-major (K = N
// pixels): the UMMA computes D[m][n] = sum_k A[m][k] B[n][k] = (A^T B)[m][n]
// directly.  These are the Gram products of Algorithm 1 (Omega^T Omega,
// Omega^T Y, Y^T Y: one launch, so each K range of Omega and Y is read from
// DRAM once and served to the tiles that share it from L2) and the U^T U of
// the stored factor: 2 N ell^2 flops over 2 N ell bytes per operand, i.e.
// HBM bound once the multiply runs on tensor cores.
//
// The output is cut into tiles of 128 rows x BN <= 256 columns; a product of
// an operand with itself keeps only the tiles that reach the diagonal.  CTA
// (tile, split) accumulates its tile over one split of the K range:
//   warp 0      TMA producer: 64-pixel K blocks of A (128 x 64) and B (BN x 64)
//               into a 4-stage ring, 128B swizzle, mbarrier transaction counts;
//               rows past an operand's last column are zero-filled by TMA
//   warp 1      MMA issuer: one elected thread, 4 x tcgen05.mma (K = 16) per
//               stage, tcgen05.commit frees the stage / signals the result
//   warp 2      TMEM allocation (BN columns, power of two >= 32)
//   warps 4-7   epilogue: tcgen05.ld 32x32b.x16 of its 32-lane quarter, fp32
//               partial tile to global, column-major within the tile (a warp
//               store covers 32 consecutive rows); the splits are summed in
//               float64, in a fixed order, by gram_tiles_reduce_kernel.
// The splits are the slowest grid index, so the tiles of one K range run
// side by side.  Every mbarrier wait is bounded: on time-out the kernel
// records an error, stops issuing, drains its own TMA copies and MMAs, frees
// TMEM and returns.
#include "internal.cuh"
#include "tma.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

namespace nys {
namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;           // bf16 elements per 128-byte swizzle row
constexpr int TC_STAGES = 4;
// every TMA x coordinate below is a multiple of TC_BK (k blocks, padded
// widths) or of 64 pixels (tile origins), so with bf16 it starts on a
// 16-byte boundary as the tiled bulk copy requires
static_assert(TC_BK % 8 == 0 && TC_BM % 64 == 0, "TMA x coordinates must be multiples of 8 bf16 values");

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand tile with rows of 128 bytes (64 bf16) written by TMA with
// 128-byte swizzle: 8-row atoms of 1024 bytes (stride-dimension offset), the
// leading offset unused for this layout (encoded 1), descriptor version 1,
// layout type 2 = SWIZZLE_128B.  The tile base is 1024-byte aligned.
__device__ __forceinline__ uint64_t sw128_kmajor_desc(const void* tile) {
    const uint32_t a = smem_u32(tile);
    return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// instruction descriptor, kind::f16: D fp32, A and B bf16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// tile table of one multi-product launch: x = source of A (bit 0), source
// of B (bit 1), product index (bits 2+); y = first row; z = first column
constexpr int GRAM_MAX_TILES = 128;
constexpr int GRAM_MAX_JOBS = 4;
struct GramTiles {
    int n;
    int4 t[GRAM_MAX_TILES];
};
struct GramJobs {
    int n;
    double* C[GRAM_MAX_JOBS];
    int ldc[GRAM_MAX_JOBS], p[GRAM_MAX_JOBS], q[GRAM_MAX_JOBS], sym[GRAM_MAX_JOBS];
};

__global__ void __launch_bounds__(256, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                   const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1,
                   const __grid_constant__ GramTiles tiles, int BN, int tmem_cols, int kblocks_total,
                   int kblocks_per_split, float* __restrict__ part, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t a_bytes = TC_BM * TC_BK * 2;
    const uint32_t b_bytes = (uint32_t)BN * TC_BK * 2;
    unsigned char* sA = base;
    unsigned char* sB = base + TC_STAGES * a_bytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + TC_STAGES * b_bytes);
    uint64_t* empty = full + TC_STAGES;
    uint64_t* accum = empty + TC_STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
    int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x;
    const int4 tl = tiles.t[tile];
    const CUtensorMap* mA = (tl.x & 1) ? &tmA1 : &tmA0;
    const CUtensorMap* mB = (tl.x & 2) ? &tmB1 : &tmB0;
    const int m0 = tl.y, n0 = tl.z;
    const int split = blockIdx.y;
    const int kb0 = split * kblocks_per_split;
    const int nk = max(0, min(kblocks_total, kb0 + kblocks_per_split) - kb0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer
        int issued = 0;
        for (int i = 0; i < nk; ++i) {
            const int s = i % TC_STAGES;
            const uint32_t ph = (uint32_t)(i / TC_STAGES) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u) || *(volatile int*)abort_flag) {
                atomicExch(err, 1);
                *(volatile int*)abort_flag = 1;
                break;
            }
            mbar_arrive_expect_tx(&full[s], a_bytes + b_bytes);
            const int kx = (kb0 + i) * TC_BK;
            tma_load_2d(sA + s * a_bytes, mA, &full[s], kx, m0);
            tma_load_2d(sB + s * b_bytes, mB, &full[s], kx, n0);
            ++issued;
        }
        // drain: every issued copy has landed before the CTA may exit
        for (int i = max(0, issued - TC_STAGES); i < issued; ++i)
            if (!mbar_wait(&full[i % TC_STAGES], (uint32_t)(i / TC_STAGES) & 1u)) atomicExch(err, 1);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = idesc_bf16(TC_BM, BN);
        for (int i = 0; i < nk; ++i) {
            const int s = i % TC_STAGES;
            const uint32_t ph = (uint32_t)(i / TC_STAGES) & 1u;
            if (!mbar_wait(&full[s], ph) || *(volatile int*)abort_flag) {
                atomicExch(err, 1);
                *(volatile int*)abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint64_t da = sw128_kmajor_desc(sA + s * a_bytes);
            const uint64_t db = sw128_kmajor_desc(sB + s * b_bytes);
#pragma unroll
            for (int k = 0; k < TC_BK / 16; ++k) {
                // +32 bytes (16 bf16) along K inside the swizzled row: +2 in the encoded address
                const uint32_t acc = (i > 0 || k > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da + 2 * k), "l"(db + 2 * k), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        // result ready (also issued after an abort, so the epilogue never waits on a dead barrier)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(accum))
                     : "memory");
    } else if (warp >= 4) {
        // epilogue: this warp's quarter of the 128 TMEM lanes = rows of the tile
        const int quarter = warp & 3;
        const bool ok = mbar_wait(accum, 0);
        tc_fence_after();
        if (!ok) atomicExch(err, 1);
        const int r = quarter * 32 + lane;
        float* out = part + ((size_t)split * tiles.n + tile) * (size_t)BN * TC_BM;
        if (ok && nk > 0 && !*(volatile int*)abort_flag) {
            for (int c0 = 0; c0 < BN; c0 += 16) {
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) out[(size_t)(c0 + j) * TC_BM + r] = __uint_as_float(v[j]);
            }
        } else if (nk == 0) {
            for (int c = 0; c < BN; ++c) out[(size_t)c * TC_BM + r] = 0.0f;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 2)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// C_job[m0 + r][n0 + c] = sum over splits (float64, fixed order) of the tile's
// partials; a product of an operand with itself writes each entry on or above
// the diagonal and its mirror.  Grid (tiles, entries / 256): one entry per
// thread.
__global__ void __launch_bounds__(256) gram_tiles_reduce_kernel(const float* __restrict__ part, int splits, int BN,
                                                                const __grid_constant__ GramTiles tiles,
                                                                const __grid_constant__ GramJobs jobs) {
    const int tile = blockIdx.x;
    const int4 tl = tiles.t[tile];
    const int job = tl.x >> 2;
    double* C = jobs.C[job];
    const int ldc = jobs.ldc[job], p = jobs.p[job], q = jobs.q[job], sym = jobs.sym[job];
    const size_t stride = (size_t)tiles.n * BN * TC_BM;
    const float* base = part + (size_t)tile * BN * TC_BM;
    for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < BN * TC_BM; e += gridDim.y * blockDim.x) {
        const int c = e / TC_BM, r = e - c * TC_BM;
        const int i = tl.y + r, j = tl.z + c;
        if (i >= p || j >= q || (sym && j < i)) continue;
        // four independent partial sums (loads in flight), combined in a fixed order
        double s4[4] = {0.0, 0.0, 0.0, 0.0};
        int z = 0;
        for (; z + 4 <= splits; z += 4)
#pragma unroll
            for (int u = 0; u < 4; ++u) s4[u] += (double)base[(size_t)(z + u) * stride + e];
        for (; z < splits; ++z) s4[0] += (double)base[(size_t)z * stride + e];
        const double s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
        C[(size_t)i * ldc + j] = s;
        if (sym) C[(size_t)j * ldc + i] = s;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn(nys_ctx* ctx) {
    static std::mutex mu;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::lock_guard<std::mutex> g(mu);
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
    }
    (void)ctx;
    return fn;
}

bool make_map(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* m, const void* ptr, int64_t N, int rows,
              int box_rows) {
    cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)N * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// The Gram products `jobs` of at most two bf16 operands (srcs[0], srcs[1],
// cols[] columns of N pixels each) in one launch.  Returns NYS_EINVAL
// (without touching the device) when the shapes are not supported, so the
// caller can take the CUDA-core path.
int gram_tc_jobs(nys_ctx* ctx, const void* const* srcs, const int* cols, int nsrc, int64_t N, int njobs,
                 const GramJob* jl) {
    if (nsrc < 1 || nsrc > 2 || njobs < 1 || njobs > GRAM_MAX_JOBS || N < TC_BK || (N % 8) != 0 ||
        N > (int64_t)0x7fffffff)
        return NYS_EINVAL;
    for (int s = 0; s < nsrc; ++s)
        if (!srcs[s] || cols[s] < 1 || cols[s] > 1024 || ((uintptr_t)srcs[s] & 15)) return NYS_EINVAL;
    auto enc = encode_fn(ctx);
    if (!enc) return NYS_EINVAL;
    // one column-tile width for the launch: at most 256, balanced over the
    // widest product's columns
    int qmax = 1;
    for (int k = 0; k < njobs; ++k) {
        if (jl[k].a < 0 || jl[k].a >= nsrc || jl[k].b < 0 || jl[k].b >= nsrc) return NYS_EINVAL;
        qmax = std::max(qmax, cols[jl[k].b]);
    }
    const int nct_max = (qmax + 255) / 256;
    const int BN = ((((qmax + nct_max - 1) / nct_max) + 15) / 16) * 16;
    int tmem_cols = 32;
    while (tmem_cols < BN) tmem_cols <<= 1;
    GramTiles tiles = {};
    GramJobs jobs = {};
    jobs.n = njobs;
    for (int k = 0; k < njobs; ++k) {
        const int p = cols[jl[k].a], q = cols[jl[k].b];
        const bool sym = jl[k].a == jl[k].b;
        jobs.C[k] = jl[k].C;
        jobs.ldc[k] = jl[k].ldc;
        jobs.p[k] = p;
        jobs.q[k] = q;
        jobs.sym[k] = sym ? 1 : 0;
        for (int m0 = 0; m0 < p; m0 += TC_BM)
            for (int n0 = 0; n0 < q; n0 += BN) {
                // a product with itself: skip tiles entirely below the diagonal
                if (sym && std::min(n0 + BN, q) - 1 < m0) continue;
                if (tiles.n >= GRAM_MAX_TILES) return NYS_EINVAL;
                tiles.t[tiles.n++] = make_int4(jl[k].a | (jl[k].b << 1) | (k << 2), m0, n0, 0);
            }
    }
    CUtensorMap mA[2], mB[2];
    for (int s = 0; s < 2; ++s) {
        const int src = s < nsrc ? s : 0;
        if (!make_map(enc, &mA[s], srcs[src], N, cols[src], TC_BM) || !make_map(enc, &mB[s], srcs[src], N, cols[src], BN))
            return NYS_EINVAL;
    }
    const int kblocks = (int)((N + TC_BK - 1) / TC_BK);
    // about one CTA per SM (each holds up to ~200 KB of shared memory)
    int splits = std::max(1, std::min(kblocks, ctx->sm_count / tiles.n));
    const int kper = (kblocks + splits - 1) / splits;
    splits = (kblocks + kper - 1) / kper;
    if (splits > 65535) return NYS_EINVAL;
    int st;
    float* part = (float*)scratch(ctx, SLOT_GRAM, (size_t)splits * tiles.n * BN * TC_BM * sizeof(float) + 64, &st);
    if (st) return st;
    int* err = (int*)scratch(ctx, SLOT_TCERR, 64, &st);
    if (st) return st;
    const size_t smem = 1024 + (size_t)TC_STAGES * (TC_BM * TC_BK * 2 + (size_t)BN * TC_BK * 2) + 256;
    if ((st = smem_optin(ctx, (const void*)gram_tc_kernel, smem))) return st;
    cudaStream_t s = ctx->stream;
    NYS_CK(ctx, cudaMemsetAsync(err, 0, sizeof(int), s));
    gram_tc_kernel<<<dim3(tiles.n, splits), 256, smem, s>>>(mA[0], mA[1], mB[0], mB[1], tiles, BN, tmem_cols, kblocks,
                                                            kper, part, err);
    NYS_LAUNCH_CK(ctx);
    gram_tiles_reduce_kernel<<<dim3(tiles.n, (BN * TC_BM + 255) / 256), 256, 0, s>>>(part, splits, BN, tiles, jobs);
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

// C (p x q, float64, ld = ldc) = A^T B for bf16 operands on tensor cores
// (A == B: one operand, the symmetric tiles only).
int gram_AtB_tc(nys_ctx* ctx, const void* A, int p, const void* B, int q, int64_t N, double* C, int ldc) {
    if (A == B && p == q) {
        const void* srcs[1] = {A};
        const int cols[1] = {p};
        const GramJob j = {0, 0, C, ldc};
        return gram_tc_jobs(ctx, srcs, cols, 1, N, 1, &j);
    }
    const void* srcs[2] = {A, B};
    const int cols[2] = {p, q};
    const GramJob j = {0, 1, C, ldc};
    return gram_tc_jobs(ctx, srcs, cols, 2, N, 1, &j);
}

}  // namespace nys

// ---------------------------------------------------------------------------
// U = (Y + v Omega) W on tcgen05, as the plain product U = [Y | Omega] W' with
// W' = [W; v W] (no elementwise pass over the tall data).  Per CTA one
// 128-pixel tile of U and one block of BN <= 256 of its q <= 1024 columns
// (the column blocks of a pixel tile are adjacent in the grid, so the tile's
// Y and Omega rows come from L2 after the first block):
//   A (128 pixels x 64 k) comes from Y or Omega, whose rows are images, so the
//     operand is MN-major: two 64-pixel TMA boxes (128B swizzle) side by side,
//     the second at LBO = 8 KB, 8-row K groups 1 KB apart (SBO)
//   B (q x 64 k) from W'^T, K-major, as in the Gram kernel
//   D in TMEM: lane = pixel, column = output column j; the epilogue writes
//     U[j][pixel] with 32 consecutive pixels per warp store.
namespace nys {
namespace {

constexpr uint32_t idesc_bf16_amn(int M, int N) { return idesc_bf16(M, N) | (1u << 15); }

__device__ __forceinline__ uint64_t sw128_mnmajor_desc(const void* tile, uint32_t lbo_bytes) {
    const uint32_t a = smem_u32(tile);
    return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)(lbo_bytes >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// W' = [W; v W] as a bf16 pair W' = hi + lo (error ~2^-16 relative), stored
// K-major: Wt[j][k] = hi, Wt[j][Kpad + k] = lo, for k < L1 from W[k][j]
// (k < ell) and for L1 <= k < 2 L1 from v W[k - L1][j]; zero padding.
constexpr int TALL_STAGES = 3;
__global__ void wt_kernel(const double* __restrict__ W, int ell, const double* __restrict__ v_dev, int L1,
                          __nv_bfloat16* __restrict__ Wt) {
    const int Kpad = 2 * L1;
    const double v = v_dev ? *v_dev : 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ell * Kpad; t += gridDim.x * blockDim.x) {
        const int j = t / Kpad, k = t - j * Kpad;
        double w = 0.0;
        if (k < L1) w = (k < ell) ? W[(size_t)k * ell + j] : 0.0;
        else w = (k - L1 < ell) ? v * W[(size_t)(k - L1) * ell + j] : 0.0;
        const __nv_bfloat16 hi = __float2bfloat16_rn((float)w);
        const __nv_bfloat16 lo = __float2bfloat16_rn((float)(w - (double)__bfloat162float(hi)));
        Wt[(size_t)j * 2 * Kpad + k] = hi;
        Wt[(size_t)j * 2 * Kpad + Kpad + k] = lo;
    }
}

template <class TO>
__global__ void __launch_bounds__(256, 1)
    tall_tc_kernel(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmO,
                   const __grid_constant__ CUtensorMap tmW, int64_t N, int q, int BN, int tmem_cols, int kb_half, int kpad, int nst,
                   TO* __restrict__ U, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t half_bytes = 64 * TC_BK * 2;          // one 64-pixel x 64-k box
    const uint32_t a_bytes = 2 * half_bytes;
    const uint32_t bh_bytes = (uint32_t)BN * TC_BK * 2;   // one of the hi / lo tiles
    const uint32_t b_bytes = 2 * bh_bytes;
    unsigned char* sA = base;
    unsigned char* sB = base + nst * a_bytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + nst * b_bytes);
    uint64_t* empty = full + nst;
    uint64_t* accum = empty + nst;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
    int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.y * TC_BM;
    const int n0 = blockIdx.x * BN;
    const int nk = 2 * kb_half;

    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        int issued = 0;
        for (int i = 0; i < nk; ++i) {
            const int s = i % nst;
            const uint32_t ph = (uint32_t)(i / nst) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u) || *(volatile int*)abort_flag) {
                atomicExch(err, 1);
                *(volatile int*)abort_flag = 1;
                break;
            }
            mbar_arrive_expect_tx(&full[s], a_bytes + b_bytes);
            const CUtensorMap* mx = (i < kb_half) ? &tmY : &tmO;
            const int krow = (i < kb_half ? i : i - kb_half) * TC_BK;
            tma_load_2d(sA + s * a_bytes, mx, &full[s], (int)m0, krow);
            tma_load_2d(sA + s * a_bytes + half_bytes, mx, &full[s], (int)m0 + 64, krow);
            tma_load_2d(sB + s * b_bytes, &tmW, &full[s], i * TC_BK, n0);
            tma_load_2d(sB + s * b_bytes + bh_bytes, &tmW, &full[s], kpad + i * TC_BK, n0);
            ++issued;
        }
        for (int i = max(0, issued - nst); i < issued; ++i)
            if (!mbar_wait(&full[i % nst], (uint32_t)(i / nst) & 1u)) atomicExch(err, 1);
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = idesc_bf16_amn(TC_BM, BN);
        for (int i = 0; i < nk; ++i) {
            const int s = i % nst;
            const uint32_t ph = (uint32_t)(i / nst) & 1u;
            if (!mbar_wait(&full[s], ph) || *(volatile int*)abort_flag) {
                atomicExch(err, 1);
                *(volatile int*)abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint64_t da = sw128_mnmajor_desc(sA + s * a_bytes, half_bytes);
            const uint64_t dbh = sw128_kmajor_desc(sB + s * b_bytes);
            const uint64_t dbl = sw128_kmajor_desc(sB + s * b_bytes + bh_bytes);
#pragma unroll
            for (int k = 0; k < TC_BK / 16; ++k) {
                // A: +16 K rows = 2048 bytes (2 swizzle atoms); B: +32 bytes inside the row.
                // Two MMAs per K step: the hi and the lo part of W'.
                const uint32_t acc = (i > 0 || k > 0) ? 1u : 0u;
                const uint64_t dak = da + (uint64_t)(k * (2048 >> 4));
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(dak), "l"(dbh + 2 * k), "r"(idesc), "r"(acc)
                    : "memory");
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(dak), "l"(dbl + 2 * k), "r"(idesc), "r"(1u)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(accum))
                     : "memory");
    } else if (warp >= 4) {
        const int quarter = warp & 3;
        const bool ok = mbar_wait(accum, 0);
        tc_fence_after();
        if (!ok) atomicExch(err, 1);
        const int64_t pix = m0 + quarter * 32 + lane;
        if (ok && !*(volatile int*)abort_flag) {
            for (int c0 = 0; c0 < BN; c0 += 16) {
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (pix < N) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (n0 + c0 + j < q) stf(U + (size_t)(n0 + c0 + j) * N + pix, __uint_as_float(v[j]));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 2)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

bool make_map_box(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* m, const void* ptr, int64_t inner,
                  int64_t rows, int box_inner, int box_rows) {
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)inner * 2};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// out (q = ell columns of N, dtype out_dt) = (Y + v Omega) W for bf16 Y, Omega;
// W is ell x ell float64 (row-major), v read from v_dev.  NYS_EINVAL when the
// shape is not supported (caller falls back to CUDA cores).
int gemm_tall_tc(nys_ctx* ctx, const void* Y, const void* Om, const double* v_dev, int64_t N, int ell,
                 const double* W, int out_dt, void* out) {
    if (ell < 1 || ell > 1024 || N < 128 || (N % 8) != 0 || N > (int64_t)0x7fffffff ||
        (N + TC_BM - 1) / TC_BM > 65535 || (((uintptr_t)Y | (uintptr_t)Om) & 15) ||
        (out_dt != NYS_BF16 && out_dt != NYS_F32))
        return NYS_EINVAL;
    auto enc = encode_fn(ctx);
    if (!enc) return NYS_EINVAL;
    const int q = ell;
    // column blocks of at most 256, balanced
    const int nct = (q + 255) / 256;
    const int BN = ((((q + nct - 1) / nct) + 15) / 16) * 16;
    int tmem_cols = 32;
    while (tmem_cols < BN) tmem_cols <<= 1;
    const int L1 = ((ell + TC_BK - 1) / TC_BK) * TC_BK;
    const int Kpad = 2 * L1;
    int st;
    __nv_bfloat16* Wt = (__nv_bfloat16*)scratch(ctx, SLOT_MISC, (size_t)q * 2 * Kpad * 2 + 256, &st);
    if (st) return st;
    int* err = (int*)scratch(ctx, SLOT_TCERR, 64, &st);
    if (st) return st;
    CUtensorMap mY, mO, mW;
    if (!make_map_box(enc, &mY, Y, N, ell, 64, TC_BK) || !make_map_box(enc, &mO, Om, N, ell, 64, TC_BK) ||
        !make_map_box(enc, &mW, Wt, 2 * Kpad, q, TC_BK, BN))
        return NYS_EINVAL;
    cudaStream_t s = ctx->stream;
    wt_kernel<<<64, 256, 0, s>>>(W, ell, v_dev, L1, Wt);
    NYS_LAUNCH_CK(ctx);
    // as many stages (2 or 3) as fit in the 227 KB shared-memory budget
    const size_t stage_bytes = 2 * 64 * TC_BK * 2 + 2 * (size_t)BN * TC_BK * 2;
    const int nst = (int)std::min<size_t>(TALL_STAGES, (227 * 1024 - 2048) / stage_bytes);
    if (nst < 2) return NYS_EINVAL;
    const size_t smem = 1024 + (size_t)nst * stage_bytes + 256;
    const dim3 grid((unsigned)nct, (unsigned)((N + TC_BM - 1) / TC_BM));
    if (out_dt == NYS_BF16) {
        if (int st2 = smem_optin(ctx, (const void*)tall_tc_kernel<__nv_bfloat16>, smem)) return st2;
        tall_tc_kernel<__nv_bfloat16><<<grid, 256, smem, s>>>(mY, mO, mW, N, q, BN, tmem_cols, L1 / TC_BK, Kpad, nst,
                                                               (__nv_bfloat16*)out, err);
    } else {
        if (int st2 = smem_optin(ctx, (const void*)tall_tc_kernel<float>, smem)) return st2;
        tall_tc_kernel<float><<<grid, 256, smem, s>>>(mY, mO, mW, N, q, BN, tmem_cols, L1 / TC_BK, Kpad, nst,
                                                       (float*)out, err);
    }
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

}  // namespace nys
