// Cholesky factorisation of the small float64 matrices of Algorithm 1 (the
// shifted core, steps 4-5) and of the preconditioner set-up (I + Ubar^T
// Ubar) on a cluster of 16 CTAs.
//
// GB300's float64 pipe issues about two FMAs per clock per SM, so the n^3/6
// FMAs of a Cholesky of n = 400 take milliseconds on one SM; spread over the
// 16 SMs of a cluster they take a tenth of that.  Columns j of the upper
// factor R (A = R^T R; row j of the lower factor L = R^T) are cut into 32
// blocks of b; CTA c holds blocks c and 31 - c (balanced work) in shared
// memory.  Right-looking by panels (one block each): the panel's owner
// factors its b x b diagonal block, every CTA solves for the panel's rows of
// its later columns, then updates those columns with the panel's rows
// gathered from the other CTAs (distributed shared memory); two cluster
// barriers per panel.  A non-positive (or non-finite) pivot is broadcast to
// every CTA before the barrier that follows it, so that all leave or retry
// together; there are no spin waits.
//
//   mode 0  A = src (n x n, row-major, ld), status in info[slot]
//   mode 1  A = sym(Omega^T Y) + v Omega^T Omega from the Gram G2 of
//           [Omega | Y] (ld 2n), v = eps sqrt(trace Omega^T Omega), times 10
//           after each failure, at most max_retries times; info[0] = status,
//           info[1] = v, info[2] = retries (as the one-CTA kernel)
// Output: L (n x n, row-major, ld n), lower triangular with zeros above.
#include "internal.cuh"
#include "chol_panel.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace nys {
namespace {

constexpr int CC = 16;           // CTAs per cluster
constexpr int CH_THREADS = 512;

__global__ void __launch_bounds__(CH_THREADS, 1)
    chol_cluster_kernel(const double* __restrict__ src, int ld, int n, int mode, double eps, int max_retries,
                        double* __restrict__ L, double* __restrict__ info, int slot, int b) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int npad = 2 * CC * b;
    extern __shared__ __align__(16) double ch_smem[];
    double* own = ch_smem;                               // [2][b][npad]: columns of R
    double* stage = own + 2 * (size_t)b * npad;          // b*b + b*npad
    __shared__ int bad_flag;
    __shared__ double sh[32];
    const int blk[2] = {rank, 2 * CC - 1 - rank};
    auto col = [&](int s, int c) { return own + ((size_t)s * b + c) * npad; };

    double v = 0.0;
    if (mode == 1) {
        double tr = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) tr += src[(size_t)i * ld + i];
        tr = block_sum(tr, sh);
        v = eps * sqrt(tr);
    }
    int retries = 0;
    bool ok = false;
    for (int attempt = 0; attempt <= (mode == 1 ? max_retries : 0); ++attempt) {
        // load: R's column j starts as A's row j (A symmetric), pad with the identity
        for (int s = 0; s < 2; ++s)
            for (int t = threadIdx.x; t < b * npad; t += blockDim.x) {
                const int c = t / npad, i = t - c * npad;
                const int j = blk[s] * b + c;
                double a;
                if (i < n && j < n) {
                    if (mode == 1) {
                        const int l2 = 2 * n;
                        const double oy = 0.5 * (src[(size_t)j * l2 + n + i] + src[(size_t)i * l2 + n + j]);
                        a = oy + v * src[(size_t)j * l2 + i];
                    } else {
                        a = src[(size_t)j * ld + i];
                    }
                } else {
                    a = (i == j) ? 1.0 : 0.0;
                }
                col(s, c)[i] = a;
            }
        if (threadIdx.x == 0) bad_flag = 0;
        cluster.sync();
        bool bad = false;
        for (int k = 0; k < 2 * CC; ++k) {
            const int owner = k < CC ? k : 2 * CC - 1 - k;
            const int oseat = k < CC ? 0 : 1;
            const int p0 = k * b;
            if (rank == owner) {
                // the b x b diagonal block by one warp (b <= 16, registers and shuffles)
                if ((threadIdx.x >> 5) == 0) {
                    const bool okb = warp_chol_block<double>([&](int c) { return col(oseat, c); }, p0, b);
                    if (!okb && (threadIdx.x & 31) == 0) bad_flag = 1;
                }
                __syncthreads();
                if (bad_flag && threadIdx.x < CC) *cluster.map_shared_rank(&bad_flag, (int)threadIdx.x) = 1;
            }
            cluster.sync();
            if (bad_flag) {
                bad = true;
                break;
            }
            {
                const double* ob = cluster.map_shared_rank(own, owner) + (size_t)oseat * b * npad;
                for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
                    const int c = e / b, i = e - c * b;
                    stage[e] = ob[(size_t)c * npad + p0 + i];   // R(p0 + i, p0 + c)
                }
            }
            __syncthreads();
            // forward substitution, one thread per column (a chain of b^2 / 2
            // FMAs is shorter than b rounds of float64 warp reductions)
            for (int q2 = threadIdx.x; q2 < 2 * b; q2 += blockDim.x) {
                const int s = q2 / b, c = q2 - s * b;
                if (blk[s] <= k) continue;
                panel_forward_subst(col(s, c), stage, p0, b);
            }
            cluster.sync();
            const int m0 = p0 + b;
            const int nm = npad - m0;
            if (nm > 0) {
                double* rows = stage + (size_t)b * b;
                for (int e = threadIdx.x; e < b * nm; e += blockDim.x) {
                    const int m = m0 + e / b, i = e - (e / b) * b;
                    const int kb = m / b, c = m - kb * b;
                    const int orank = kb < CC ? kb : 2 * CC - 1 - kb, os = kb < CC ? 0 : 1;
                    const double* ob = cluster.map_shared_rank(own, orank) + ((size_t)os * b + c) * npad;
                    rows[(size_t)(m - m0) * b + i] = ob[p0 + i];
                }
                __syncthreads();
                for (int s = 0; s < 2; ++s) {
                    if (blk[s] <= k) continue;
                    for (int e = threadIdx.x; e < b * npad; e += blockDim.x) {
                        const int c = e / npad, i = e - c * npad;
                        const int j = blk[s] * b + c;
                        if (i < m0 || i > j) continue;
                        double* cc = col(s, c);
                        double acc = 0.0;
                        for (int t = 0; t < b; ++t) acc += rows[(size_t)(i - m0) * b + t] * cc[p0 + t];
                        cc[i] -= acc;
                    }
                }
            }
            __syncthreads();
        }
        // all CTAs agree on `bad` (each read its own copy after the same barrier)
        if (!bad) {
            ok = true;
            retries = attempt;
            break;
        }
        retries = attempt;
        if (mode == 1) v *= 10.0;
        // no CTA reloads its columns before every CTA has stopped reading them
        cluster.sync();
    }
    if (ok) {
        for (int s = 0; s < 2; ++s)
            for (int t = threadIdx.x; t < b * n; t += blockDim.x) {
                const int c = t / n, i = t - c * n;
                const int j = blk[s] * b + c;
                if (j < n) L[(size_t)j * n + i] = i <= j ? col(s, c)[i] : 0.0;
            }
    }
    if (rank == 0 && threadIdx.x == 0) {
        if (mode == 1) {
            info[0] = ok ? 0.0 : 1.0;
            info[1] = ok ? v : v / 10.0;
            info[2] = (double)retries;
        } else {
            info[slot] = ok ? 0.0 : 1.0;
        }
    }
    // no CTA leaves while another may still read its shared memory
    cluster.sync();
}

}  // namespace

// L = chol(A) by the cluster kernel (see above); NYS_EINVAL (nothing
// launched) when n is outside [48, 512] or the cluster cannot be placed.
int chol_cluster(nys_ctx* ctx, const double* src, int ld, int n, int mode, double eps, int max_retries, double* L,
                 double* info, int slot) {
    if (n < 48 || n > 512) return NYS_EINVAL;
    const int b = (n + 2 * CC - 1) / (2 * CC);
    const int npad = 2 * CC * b;
    const size_t smem = (2 * (size_t)b * npad + (size_t)b * b + (size_t)b * npad) * sizeof(double) + 64;
    if (smem > 220 * 1024) return NYS_EINVAL;
    auto k = chol_cluster_kernel;
    NYS_CK(ctx, cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    if (int st = smem_optin(ctx, (const void*)k, smem)) return st;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CC, 1, 1);
    cfg.blockDim = dim3(CH_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k, &cfg) != cudaSuccess || clusters < 1) {
        cudaGetLastError();
        return NYS_EINVAL;
    }
    NYS_CK(ctx, cudaLaunchKernelEx(&cfg, k, src, ld, n, mode, eps, max_retries, L, info, slot, b));
    ++ctx->launches;
    return NYS_OK;
}

}  // namespace nys
