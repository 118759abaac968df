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
#include "internal.cuh"

#include <cmath>

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

// forward: one CTA per (angle, image); threads over detector bins
template <class TI, class TO, class TC>
__global__ void __launch_bounds__(256) radon_fwd_kernel(const TI* __restrict__ x, TO* __restrict__ y, int n1, int n2,
                                                        int n_angles, int n_bins, RTab<TC> tab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int k = blockIdx.x;
    const int b = blockIdx.y;
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
    const TI* xb = x + (size_t)b * n1 * n2;
    // element (line l, position p): row-step -> x[l][p], column-step -> x[p][l]
    const int sl = rs ? n2 : 1, sp = rs ? 1 : n2;
    const TC wt = tab.wt[k];
    for (int m = threadIdx.x; m < n_bins; m += blockDim.x) {
        const int qi = tab.qi[(size_t)k * n_bins + m];
        const TC qf = tab.qf[(size_t)k * n_bins + m];
        TC acc = TC(0);
        for (int l = 0; l < nl; ++l) {
            int lo;
            TC w;
            sample_pos<TC>(qi, qf, s_ri[l], s_rf[l], lo, w);
            const TI* row = xb + (size_t)l * sl;
            if (lo >= 0 && lo < na) acc = fma(TC(1) - w, (TC)ldf(row + (size_t)lo * sp), acc);
            if (lo + 1 >= 0 && lo + 1 < na) acc = fma(w, (TC)ldf(row + (size_t)(lo + 1) * sp), acc);
        }
        stf(y + ((size_t)b * n_angles + k) * n_bins + m, wt * acc);
    }
}

// adjoint: one thread per pixel, loop over all angles; for each angle the
// rays through the pixel's line that land within one position of the pixel
// are found from the continuous bin m* = c_b + slope (p - c - R_l) and the four
// integer candidates around it are tested with the forward's exact test.
template <class TI, class TO, class TC>
__global__ void __launch_bounds__(256) radon_adj_kernel(const TI* __restrict__ s, TO* __restrict__ x, int n1, int n2,
                                                        int n_angles, int n_bins, RTab<TC> tab, TC c1, TC c2,
                                                        TC cb) {
    const int j = blockIdx.x * 16 + (threadIdx.x & 15);
    const int i = blockIdx.y * 16 + (threadIdx.x >> 4);
    const int b = blockIdx.z;
    if (i >= n1 || j >= n2) return;
    const TI* sb = s + (size_t)b * n_angles * n_bins;
    TC acc = TC(0);
    for (int k = 0; k < n_angles; ++k) {
        const int rs = tab.rowstep[k];
        const int l = rs ? i : j;          // line of this pixel
        const int p = rs ? j : i;          // position along the line
        const TC cpos = rs ? c2 : c1;
        const int ri = tab.ri[(size_t)k * tab.nl_max + l];
        const TC rf = tab.rf[(size_t)k * tab.nl_max + l];
        const TC slope = tab.slope[k];
        // position u(m) = Q_m + R_l = cpos + (m - cb)/slope + R_l = p  ->  m*
        const TC mstar = cb + slope * ((TC)p - cpos - ((TC)ri + rf));
        const int m0 = (int)floor(mstar) - 1;
        TC part = TC(0);
#pragma unroll
        for (int dm = 0; dm < 4; ++dm) {
            const int m = m0 + dm;
            if (m < 0 || m >= n_bins) continue;
            int lo;
            TC w;
            sample_pos<TC>(tab.qi[(size_t)k * n_bins + m], tab.qf[(size_t)k * n_bins + m], ri, rf, lo, w);
            TC wgt = TC(0);
            if (lo == p) wgt = TC(1) - w;
            else if (lo + 1 == p) wgt = w;
            if (wgt != TC(0)) part = fma(wgt, (TC)ldf(sb + (size_t)k * n_bins + m), part);
        }
        acc = fma(tab.wt[k], part, acc);
    }
    stf(x + ((size_t)b * n1 + i) * n2 + j, acc);
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
    std::vector<TC> qf((size_t)A * B), rf((size_t)A * nl_max, TC(0)), wt(A), slope(A);
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
        for (int m = 0; m < B; ++m) split<TC>(c_pos + (m - cb) / den, qi[(size_t)k * B + m], qf[(size_t)k * B + m]);
        const int nl = rs ? n1 : n2;
        for (int l = 0; l < nl; ++l)
            split<TC>(-(l - c_line) * oth / den, ri[(size_t)k * nl_max + l], rf[(size_t)k * nl_max + l]);
    }
    size_t off = 0;
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    const size_t sz_qi = al(qi.size() * 4), sz_qf = al(qf.size() * sizeof(TC)), sz_ri = al(ri.size() * 4),
                 sz_rf = al(rf.size() * sizeof(TC)), sz_a = al(A * sizeof(TC)), sz_rs = al(A * 4);
    const size_t total = sz_qi + sz_qf + sz_ri + sz_rf + 2 * sz_a + sz_rs;
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
    t.rowstep = (const int*)(base + off);
    t.nl_max = nl_max;
    return t;
}

template <class TI, class TO, class TC>
int radon_fwd(nys_op* op, const void* x, void* y, int batch) {
    const int nl_max = std::max(op->n1, op->n2);
    const size_t sm = ((nl_max + 3) & ~3) * 4 + nl_max * sizeof(TC);
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int nb = std::min(65535, batch - b0);
        dim3 grid(op->n_angles, nb);
        radon_fwd_kernel<TI, TO, TC><<<grid, 256, sm, op->ctx->stream>>>(
            (const TI*)x + (size_t)b0 * op->N, (TO*)y + (size_t)b0 * op->M, op->n1, op->n2, op->n_angles,
            op->n_bins, tables<TC>(op));
        NYS_LAUNCH_CK(op->ctx);
    }
    return NYS_OK;
}

template <class TI, class TO, class TC>
int radon_adj(nys_op* op, const void* s, void* x, int batch) {
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int nb = std::min(65535, batch - b0);
        dim3 grid((op->n2 + 15) / 16, (op->n1 + 15) / 16, nb);
        radon_adj_kernel<TI, TO, TC><<<grid, 256, 0, op->ctx->stream>>>(
            (const TI*)s + (size_t)b0 * op->M, (TO*)x + (size_t)b0 * op->N, op->n1, op->n2, op->n_angles,
            op->n_bins, tables<TC>(op), (TC)((op->n1 - 1) / 2.0), (TC)((op->n2 - 1) / 2.0),
            (TC)((op->n_bins - 1) / 2.0));
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
