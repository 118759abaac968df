// Parallel-beam ray transform A and its exact transpose A^T (Sec. IV-C, the CT
// forward model), discretised with Joseph's method (P. M. Joseph, "An improved
// algorithm for reprojecting rays through pixel images", IEEE TMI 1982).
//
// Geometry: pixel (i, j) sits at x = j - c2, y = i - c1 (c = (n-1)/2); ray
// (theta_k, t_m) is the line x cos + y sin = t with theta_k = k span / n_angles
// and t_m = m - (n_bins - 1)/2.  A "row-step" angle (|cos| + 1e-9 >= |sin|)
// samples the ray once per image row i at column position
//     u(i, m) = c2 + t_m / cos - (i - c1) tan = Q_m + R_i
// with linear interpolation between columns floor(u) and floor(u) + 1 and
// weight 1/|cos|; a "column-step" angle swaps the roles of rows and columns
// (Q_m = c1 + t_m / sin, R_j = -(j - c2) cot, weight 1/|sin|).  Samples that
// fall outside the image contribute zero.
//
// Precision: Q_m and R_l are split on the host, in float64, into an integer
// part and a fraction in [0, 1).  The device adds the two fractions (error at
// most one float ulp of a number below 2), so interpolation weights carry an
// absolute error near 1e-7 instead of the ~3e-5 that a float position near 500
// would carry.  The forward (ray-driven) and the adjoint (pixel-driven gather)
// evaluate the SAME float expressions for every (ray, line) pair, so the
// adjoint is the exact transpose of the forward up to summation order, with
// no atomics.
//
// Forward: one CTA per (angle, group of IB images), each thread three bins,
// stepping along the lines of the angle.  The image is read "line-major":
// row-step angles read the row-major image, column-step angles a transposed
// copy (made once per batch chunk), so consecutive bins of a warp read
// consecutive addresses for both kinds of angle.  The per-line table entries
// are staged in shared memory and shared by the three bins and the IB images.
// Adjoint: one CTA per (16 x 16 pixel tile, group of IB images).  Angles are
// taken AK at a time: for each, the window of bins that can reach the tile
// (from the four tile corners) is staged in shared memory with its tables and
// sinogram values, so the per-pixel candidate tests read shared memory only;
// candidates outside the window (none for |slope| <= 1, kept for safety) fall
// back to global loads.
#include "internal.cuh"

#include <cmath>
#include <type_traits>

namespace nys {
namespace {

template <class TC>
struct RTab {
    const int* qi;     // [n_angles][n_bins]
    const TC* qf;      // [n_angles][n_bins]
    const int* ri;     // [n_angles][nl_max]
    const TC* rf;      // [n_angles][nl_max]
    const TC* wt;      // [n_angles] 1/|cos| or 1/|sin|
    const TC* slope;   // [n_angles] dm/du = cos (row-step) or sin (column-step)
    const TC* oth;     // [n_angles] sin (row-step) or cos (column-step): dm*/dl
    const int* rowstep;// [n_angles]
    int nl_max;
};

template <class TC>
__device__ __forceinline__ void sample_pos(int qi, TC qf, int ri, TC rf, int& lo, TC& w) {
    TC f = qf + rf;
    const int carry = f >= TC(1) ? 1 : 0;
    f -= (TC)carry;
    lo = qi + ri + carry;
    w = f;
}

// xr (optional) / xT: line-major copies of `batch` images in the compute type;
// xT[b][j][i] = x[b][i][j]
template <class TI, class TC>
__global__ void radon_prep_kernel(const TI* __restrict__ x, TC* __restrict__ xr, TC* __restrict__ xT, int n1, int n2) {
    pdl_enter();
    __shared__ TC tile[32][33];
    const int b = blockIdx.z;
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const TI* xb = x + (size_t)b * n1 * n2;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        TC v = TC(0);
        if (i < n1 && j < n2) {
            v = (TC)ldf(xb + (size_t)i * n2 + j);
            if (xr) xr[(size_t)b * n1 * n2 + (size_t)i * n2 + j] = v;
        }
        tile[r][threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r, i = i0 + threadIdx.x;
        if (i < n1 && j < n2) xT[(size_t)b * n1 * n2 + (size_t)j * n1 + i] = tile[threadIdx.x][r];
    }
}

// forward: one CTA per (angle, IB images); threads over bins, three per thread
template <class TC, class TO, int IB>
__global__ void __launch_bounds__(256) radon_fwd2_kernel(const TC* __restrict__ xr, const TC* __restrict__ xT,
                                                         TO* __restrict__ y, int n1, int n2, int n_angles,
                                                         int n_bins, int batch, RTab<TC> tab) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int k = blockIdx.x;
    const int b0 = blockIdx.y * IB;
    const int rs = tab.rowstep[k];
    const int nl = rs ? n1 : n2;       // lines (rows for row-step)
    const int na = rs ? n2 : n1;       // positions along a line
    int* s_ri = reinterpret_cast<int*>(smem_raw);
    TC* s_rf = reinterpret_cast<TC*>(s_ri + ((nl + 3) & ~3));
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
        s_ri[l] = tab.ri[(size_t)k * tab.nl_max + l];
        s_rf[l] = tab.rf[(size_t)k * tab.nl_max + l];
    }
    __syncthreads();
    const size_t N = (size_t)n1 * n2;
    const TC* src = (rs ? xr : xT) + (size_t)b0 * N;
    const TC wt = tab.wt[k];
    for (int mb = threadIdx.x; mb < n_bins; mb += 3 * blockDim.x) {
        int qi[3];
        TC qf[3];
        bool ok[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int m = mb + c * blockDim.x;
            ok[c] = m < n_bins;
            qi[c] = ok[c] ? tab.qi[(size_t)k * n_bins + m] : 0;
            qf[c] = ok[c] ? tab.qf[(size_t)k * n_bins + m] : TC(0);
        }
        TC acc[3][IB];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 0; q < IB; ++q) acc[c][q] = TC(0);
#pragma unroll 4
        for (int l = 0; l < nl; ++l) {
            const int ri = s_ri[l];
            const TC rf = s_rf[l];
            const TC* line = src + (size_t)l * na;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                int lo;
                TC w;
                sample_pos<TC>(qi[c], qf[c], ri, rf, lo, w);
                const bool in0 = ok[c] && lo >= 0 && lo < na, in1 = ok[c] && lo + 1 >= 0 && lo + 1 < na;
#pragma unroll
                for (int q = 0; q < IB; ++q) {
                    const TC* lq = line + (size_t)q * N;
                    const bool live = b0 + q < batch;
                    const TC v0 = (in0 && live) ? lq[lo] : TC(0);
                    const TC v1 = (in1 && live) ? lq[lo + 1] : TC(0);
                    acc[c][q] = fma(TC(1) - w, v0, acc[c][q]);
                    acc[c][q] = fma(w, v1, acc[c][q]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int m = mb + c * blockDim.x;
            if (!ok[c]) continue;
#pragma unroll
            for (int q = 0; q < IB; ++q)
                if (b0 + q < batch) stf(y + ((size_t)(b0 + q) * n_angles + k) * n_bins + m, wt * acc[c][q]);
        }
    }
}

// adjoint: one CTA per (16 x 16 pixel tile, IB images), angles AK at a time.
// For a pixel at position p on line l of angle k, the rays that sample it
// are found from the continuous bin m* = c_b + slope (p - c - R_l) and the
// three integer candidates around it are tested with the forward's exact test.
constexpr int ATS = 16;     // tile side
constexpr int AWIN = 48;    // staged bins per angle
template <class TI, class TO, class TC, int IB, int AK>
__global__ void __launch_bounds__(256) radon_adj2_kernel(const TI* __restrict__ s, TO* __restrict__ x, int n1, int n2,
                                                         int n_angles, int n_bins, int batch, RTab<TC> tab, TC c1,
                                                         TC c2, TC cb) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // per-angle scalars for every angle, staged once
    int* g_rs = reinterpret_cast<int*>(smem_raw);
    TC* g_slope = reinterpret_cast<TC*>(g_rs + ((n_angles + 3) & ~3));
    TC* g_oth = g_slope + n_angles;
    TC* g_wt = g_oth + n_angles;
    __shared__ int sq_i[AK][AWIN];
    __shared__ TC sq_f[AK][AWIN];
    __shared__ TC ss[AK][IB][AWIN];
    __shared__ int sr_i[AK][ATS];
    __shared__ TC sr_f[AK][ATS];
    __shared__ int s_mlo[AK];
    const int i0 = blockIdx.y * ATS, j0 = blockIdx.x * ATS;
    const int b0 = blockIdx.z * IB;
    const int ti = threadIdx.x / ATS, tj = threadIdx.x % ATS;
    const int i = i0 + ti, j = j0 + tj;
    const bool valid = i < n1 && j < n2;
    const size_t M = (size_t)n_angles * n_bins;
    for (int k = threadIdx.x; k < n_angles; k += blockDim.x) {
        g_rs[k] = tab.rowstep[k];
        g_slope[k] = tab.slope[k];
        g_oth[k] = tab.oth[k];
        g_wt[k] = tab.wt[k];
    }
    __syncthreads();
    // window start of angle k for this tile: m* = cb + slope (p - cpos) + oth (l - cline)
    // is affine in (p, l), so its minimum over the tile is at a corner; two
    // bins of margin cover the float rounding of the split tables
    auto window = [&](int k) -> int {
        const int rs = g_rs[k];
        const TC sl = g_slope[k], ot = g_oth[k];
        const TC pa = (TC)(rs ? j0 : i0) - (rs ? c2 : c1);
        const TC la = (TC)(rs ? i0 : j0) - (rs ? c1 : c2);
        const TC mp = fmin(sl * pa, sl * (pa + TC(ATS - 1)));
        const TC ml = fmin(ot * la, ot * (la + TC(ATS - 1)));
        return (int)floor(cb + mp + ml) - 2;
    };
    TC acc[IB];
#pragma unroll
    for (int q = 0; q < IB; ++q) acc[q] = TC(0);
    for (int k0 = 0; k0 < n_angles; k0 += AK) {
        __syncthreads();   // the previous round's shared tables are consumed
        if (threadIdx.x < AK) s_mlo[threadIdx.x] = (k0 + threadIdx.x < n_angles) ? window(k0 + threadIdx.x) : 0;
        __syncthreads();
        for (int e = threadIdx.x; e < AK * AWIN; e += blockDim.x) {
            const int a = e / AWIN, w = e % AWIN;
            const int k = k0 + a;
            bool ok = k < n_angles;
            const int m = ok ? s_mlo[a] + w : 0;
            ok = ok && m >= 0 && m < n_bins;
            sq_i[a][w] = ok ? tab.qi[(size_t)k * n_bins + m] : 0;
            sq_f[a][w] = ok ? tab.qf[(size_t)k * n_bins + m] : TC(0);
#pragma unroll
            for (int q = 0; q < IB; ++q)
                ss[a][q][w] = (ok && b0 + q < batch) ? (TC)ldf(s + (size_t)(b0 + q) * M + (size_t)k * n_bins + m) : TC(0);
        }
        for (int e = threadIdx.x; e < AK * ATS; e += blockDim.x) {
            const int a = e / ATS, q = e % ATS;
            const int k = k0 + a;
            int ri = 0;
            TC rf = TC(0);
            if (k < n_angles) {
                const int rs = g_rs[k];
                const int l = (rs ? i0 : j0) + q;
                if (l < (rs ? n1 : n2)) {
                    ri = tab.ri[(size_t)k * tab.nl_max + l];
                    rf = tab.rf[(size_t)k * tab.nl_max + l];
                }
            }
            sr_i[a][q] = ri;
            sr_f[a][q] = rf;
        }
        __syncthreads();
        if (!valid) continue;
        const int na = min(AK, n_angles - k0);
        for (int a = 0; a < na; ++a) {
            const int k = k0 + a;
            const int rs = g_rs[k];
            const int lq = rs ? ti : tj;       // line of this pixel within the tile
            const int p = rs ? j : i;          // position along the line
            const TC cpos = rs ? c2 : c1;
            const int ri = sr_i[a][lq];
            const TC rf = sr_f[a][lq];
            const TC mstar = cb + g_slope[k] * ((TC)p - cpos - ((TC)ri + rf));
            // a bin m samples this pixel only if |u(m) - p| < 1, i.e. |m - m*| <
            // |slope| <= 1: the (at most three) integers in (m* - 1, m* + 1),
            // with a margin for the rounding of m*
            const int m0 = (int)ceil(mstar - TC(1) - TC(1e-4));
            const int mlo = s_mlo[a];
            TC part[IB];
#pragma unroll
            for (int q = 0; q < IB; ++q) part[q] = TC(0);
#pragma unroll
            for (int dm = 0; dm < 3; ++dm) {
                const int m = m0 + dm;
                if (m < 0 || m >= n_bins) continue;
                const int w = m - mlo;
                const bool in = w >= 0 && w < AWIN;
                int lo;
                TC wf;
                if (in) sample_pos<TC>(sq_i[a][w], sq_f[a][w], ri, rf, lo, wf);
                else sample_pos<TC>(tab.qi[(size_t)k * n_bins + m], tab.qf[(size_t)k * n_bins + m], ri, rf, lo, wf);
                TC wgt = TC(0);
                if (lo == p) wgt = TC(1) - wf;
                else if (lo + 1 == p) wgt = wf;
                if (wgt == TC(0)) continue;
#pragma unroll
                for (int q = 0; q < IB; ++q) {
                    const TC sv = in ? ss[a][q][w]
                                     : ((b0 + q < batch) ? (TC)ldf(s + (size_t)(b0 + q) * M + (size_t)k * n_bins + m)
                                                         : TC(0));
                    part[q] = fma(wgt, sv, part[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < IB; ++q) acc[q] = fma(g_wt[k], part[q], acc[q]);
        }
    }
    if (!valid) return;
#pragma unroll
    for (int q = 0; q < IB; ++q)
        if (b0 + q < batch) stf(x + ((size_t)(b0 + q) * n1 + i) * n2 + j, acc[q]);
}

template <class TC>
void split(double v, int& I, TC& F) {
    double fl = std::floor(v);
    double fr = v - fl;
    TC f = (TC)fr;
    if (f >= TC(1)) {
        f = TC(0);
        fl += 1.0;
    }
    I = (int)fl;
    F = f;
}

template <class TC>
int build_tables(nys_op* op) {
    const int A = op->n_angles, B = op->n_bins, n1 = op->n1, n2 = op->n2;
    const int nl_max = std::max(n1, n2);
    const double c1 = (n1 - 1) / 2.0, c2 = (n2 - 1) / 2.0, cb = (B - 1) / 2.0;
    std::vector<int> qi((size_t)A * B), ri((size_t)A * nl_max, 0), rowstep(A);
    std::vector<TC> qf((size_t)A * B), rf((size_t)A * nl_max, TC(0)), wt(A), slope(A), othv(A);
    for (int k = 0; k < A; ++k) {
        const double th = k * (op->span / A);
        const double cs = std::cos(th), sn = std::sin(th);
        const bool rs = std::fabs(cs) + 1e-9 >= std::fabs(sn);
        rowstep[k] = rs;
        const double c_line = rs ? c1 : c2;   // centre of the line index
        const double c_pos = rs ? c2 : c1;
        const double den = rs ? cs : sn;      // u = c_pos + t/den - (l - c_line) * other/den
        const double oth = rs ? sn : cs;
        wt[k] = (TC)(1.0 / std::fabs(den));
        slope[k] = (TC)den;
        othv[k] = (TC)oth;
        for (int m = 0; m < B; ++m) split<TC>(c_pos + (m - cb) / den, qi[(size_t)k * B + m], qf[(size_t)k * B + m]);
        const int nl = rs ? n1 : n2;
        for (int l = 0; l < nl; ++l)
            split<TC>(-(l - c_line) * oth / den, ri[(size_t)k * nl_max + l], rf[(size_t)k * nl_max + l]);
    }
    size_t off = 0;
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    const size_t sz_qi = al(qi.size() * 4), sz_qf = al(qf.size() * sizeof(TC)), sz_ri = al(ri.size() * 4),
                 sz_rf = al(rf.size() * sizeof(TC)), sz_a = al(A * sizeof(TC)), sz_rs = al(A * 4);
    const size_t total = sz_qi + sz_qf + sz_ri + sz_rf + 3 * sz_a + sz_rs;
    NYS_CK(op->ctx, cudaMalloc(&op->rtab, total));
    char* base = (char*)op->rtab;
    auto put = [&](const void* src, size_t n, size_t sz) {
        cudaError_t e = cudaMemcpy(base + off, src, n, cudaMemcpyHostToDevice);
        off += sz;
        return e;
    };
    NYS_CK(op->ctx, put(qi.data(), qi.size() * 4, sz_qi));
    NYS_CK(op->ctx, put(qf.data(), qf.size() * sizeof(TC), sz_qf));
    NYS_CK(op->ctx, put(ri.data(), ri.size() * 4, sz_ri));
    NYS_CK(op->ctx, put(rf.data(), rf.size() * sizeof(TC), sz_rf));
    NYS_CK(op->ctx, put(wt.data(), A * sizeof(TC), sz_a));
    NYS_CK(op->ctx, put(slope.data(), A * sizeof(TC), sz_a));
    NYS_CK(op->ctx, put(othv.data(), A * sizeof(TC), sz_a));
    NYS_CK(op->ctx, put(rowstep.data(), A * 4, sz_rs));
    return NYS_OK;
}

template <class TC>
RTab<TC> tables(const nys_op* op) {
    const int A = op->n_angles, B = op->n_bins;
    const int nl_max = std::max(op->n1, op->n2);
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    const char* base = (const char*)op->rtab;
    RTab<TC> t;
    size_t off = 0;
    t.qi = (const int*)(base + off);
    off += al((size_t)A * B * 4);
    t.qf = (const TC*)(base + off);
    off += al((size_t)A * B * sizeof(TC));
    t.ri = (const int*)(base + off);
    off += al((size_t)A * nl_max * 4);
    t.rf = (const TC*)(base + off);
    off += al((size_t)A * nl_max * sizeof(TC));
    t.wt = (const TC*)(base + off);
    off += al(A * sizeof(TC));
    t.slope = (const TC*)(base + off);
    off += al(A * sizeof(TC));
    t.oth = (const TC*)(base + off);
    off += al(A * sizeof(TC));
    t.rowstep = (const int*)(base + off);
    t.nl_max = nl_max;
    return t;
}

template <class TI, class TO, class TC>
int radon_fwd(nys_op* op, const void* x, void* y, int batch) {
    const int nl_max = std::max(op->n1, op->n2);
    const size_t sm = ((nl_max + 3) & ~3) * 4 + nl_max * sizeof(TC);
    const size_t N = (size_t)op->N;
    cudaStream_t st = op->ctx->stream;
    TC* xT = (TC*)op->lines;
    TC* xr = xT + (size_t)op->chunk * N;
    for (int b0 = 0; b0 < batch; b0 += op->chunk) {
        const int nb = std::min(op->chunk, batch - b0);
        const TI* xb = (const TI*)x + (size_t)b0 * N;
        // the row-major source is x itself when it already has the compute type
        const bool same = std::is_same<TI, TC>::value;
        NYS_CK(op->ctx, launch_pdl(radon_prep_kernel<TI, TC>, dim3((op->n2 + 31) / 32, (op->n1 + 31) / 32, nb),
                                   dim3(32, 8), 0, st, xb, same ? nullptr : xr, xT, op->n1, op->n2));
        NYS_LAUNCH_CK(op->ctx);
        const TC* src_r = same ? (const TC*)xb : xr;
        TO* yb = (TO*)y + (size_t)b0 * op->M;
        if (nb >= 4) {
            const int full = nb / 4 * 4;
            NYS_CK(op->ctx, launch_pdl(radon_fwd2_kernel<TC, TO, 4>, dim3(op->n_angles, full / 4), 256, sm, st, src_r,
                                       (const TC*)xT, yb, op->n1, op->n2, op->n_angles, op->n_bins, full,
                                       tables<TC>(op)));
            NYS_LAUNCH_CK(op->ctx);
            if (full < nb) {
                NYS_CK(op->ctx, launch_pdl(radon_fwd2_kernel<TC, TO, 1>, dim3(op->n_angles, nb - full), 256, sm, st,
                                           src_r + (size_t)full * N, (const TC*)(xT + (size_t)full * N),
                                           yb + (size_t)full * op->M, op->n1, op->n2, op->n_angles, op->n_bins,
                                           nb - full, tables<TC>(op)));
                NYS_LAUNCH_CK(op->ctx);
            }
        } else {
            NYS_CK(op->ctx, launch_pdl(radon_fwd2_kernel<TC, TO, 1>, dim3(op->n_angles, nb), 256, sm, st, src_r,
                                       (const TC*)xT, yb, op->n1, op->n2, op->n_angles, op->n_bins, nb,
                                       tables<TC>(op)));
            NYS_LAUNCH_CK(op->ctx);
        }
    }
    return NYS_OK;
}

template <class TI, class TO, class TC, int IB, int AK>
void radon_adj_launch(nys_op* op, const TI* s, TO* x, int nb) {
    dim3 grid((op->n2 + ATS - 1) / ATS, (op->n1 + ATS - 1) / ATS, (nb + IB - 1) / IB);
    const size_t sm = (((size_t)op->n_angles + 3) & ~size_t(3)) * 4 + 3 * (size_t)op->n_angles * sizeof(TC);
    // opt in to more than 48 KB of shared memory when the angle tables need it
    static size_t attr = 0;
    if (sm > attr) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, radon_adj2_kernel<TI, TO, TC, IB, AK>) == cudaSuccess &&
            fa.sharedSizeBytes + sm > 48 * 1024)
            cudaFuncSetAttribute(radon_adj2_kernel<TI, TO, TC, IB, AK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        attr = sm;
    }
    // a launch error is left for the caller's launch check (cudaGetLastError)
    (void)launch_pdl(radon_adj2_kernel<TI, TO, TC, IB, AK>, grid, 256, sm, op->ctx->stream, s, x, op->n1, op->n2,
                     op->n_angles, op->n_bins, nb, tables<TC>(op), (TC)((op->n1 - 1) / 2.0), (TC)((op->n2 - 1) / 2.0),
                     (TC)((op->n_bins - 1) / 2.0));
}

template <class TI, class TO, class TC>
int radon_adj(nys_op* op, const void* s, void* x, int batch) {
    for (int b0 = 0; b0 < batch; b0 += 65535 * 4) {
        const int nb = std::min(65535 * 4, batch - b0);
        const TI* sb = (const TI*)s + (size_t)b0 * op->M;
        TO* xb = (TO*)x + (size_t)b0 * op->N;
        // 4, 8 or 16 angles per round (nys_op_autotune); float64 stays at <= 8
        const int ak = (sizeof(TC) == 8 && op->radon_adj_ak > 8) ? 8 : op->radon_adj_ak;
        if (nb >= 4) {
            if (ak == 4) radon_adj_launch<TI, TO, TC, 4, 4>(op, sb, xb, nb);
            else if (ak == 16) radon_adj_launch<TI, TO, TC, 4, 16>(op, sb, xb, nb);
            else radon_adj_launch<TI, TO, TC, 4, 8>(op, sb, xb, nb);
        } else {
            if (ak == 4) radon_adj_launch<TI, TO, TC, 1, 4>(op, sb, xb, nb);
            else if (ak == 16) radon_adj_launch<TI, TO, TC, 1, 16>(op, sb, xb, nb);
            else radon_adj_launch<TI, TO, TC, 1, 8>(op, sb, xb, nb);
        }
        NYS_LAUNCH_CK(op->ctx);
    }
    return NYS_OK;
}

template <class TI, class TO, class TC>
int radon_typed(nys_op* op, int which, const void* x, void* y, int batch) {
    if (which == 0) return radon_fwd<TI, TO, TC>(op, x, y, batch);
    if (which == 1) return radon_adj<TI, TO, TC>(op, x, y, batch);
    for (int b0 = 0; b0 < batch; b0 += op->chunk) {
        const int nb = std::min(op->chunk, batch - b0);
        if (int st = radon_fwd<TI, TC, TC>(op, (const TI*)x + (size_t)b0 * op->N, op->inter, nb)) return st;
        if (int st = radon_adj<TC, TO, TC>(op, op->inter, (TO*)y + (size_t)b0 * op->N, nb)) return st;
    }
    return NYS_OK;
}

}  // namespace

int radon_setup(nys_op* op) {
    const bool f64 = op->dtype == NYS_F64;
    int st = f64 ? build_tables<double>(op) : build_tables<float>(op);
    if (st) return st;
    op->chunk = 32;
    NYS_CK(op->ctx, cudaMalloc(&op->inter, (size_t)op->chunk * op->M * (f64 ? 8 : 4)));
    // line-major copies for the forward: transposed + row-major, `chunk` images
    NYS_CK(op->ctx, cudaMalloc(&op->lines, (size_t)2 * op->chunk * op->N * (f64 ? 8 : 4)));
    return NYS_OK;
}

int radon_run(nys_op* op, int which, const void* x, void* y, int batch, int in_dt, int out_dt) {
    if (op->dtype == NYS_F64) {
        if (in_dt != NYS_F64 || out_dt != NYS_F64) return fail(op->ctx, NYS_EINVAL, "f64 operator needs f64 data");
        return radon_typed<double, double, double>(op, which, x, y, batch);
    }
    const bool ib = in_dt == NYS_BF16, ob = out_dt == NYS_BF16;
    if (!ib && !ob) return radon_typed<float, float, float>(op, which, x, y, batch);
    if (ib && ob) return radon_typed<__nv_bfloat16, __nv_bfloat16, float>(op, which, x, y, batch);
    if (ib) return radon_typed<__nv_bfloat16, float, float>(op, which, x, y, batch);
    return radon_typed<float, __nv_bfloat16, float>(op, which, x, y, batch);
}

}  // namespace nys
