// Fan-beam ray transform (the second CT geometry of the experiments) and its
// exact transpose, discretised with Joseph's method like the parallel-beam
// one.  A point source on a circle of radius R about the image centre and a
// flat detector at distance D from it: at angle theta, e_s = (cos, sin),
// e_d = (-sin, cos), source S = R e_s, detector centre S - D e_s, bin m at
// offset u_m = (m - (n_bins-1)/2) du along e_d; ray m runs from S to its bin
// along d = -D e_s + u_m e_d.  A ray with |d_y| >= |d_x| samples every row i
// at column position u = a + b i (b = d_x/d_y), weight |d|/|d_y|; any other
// ray samples every column j at row position u = a + b j (b = d_y/d_x),
// weight |d|/|d_x|; linear interpolation between floor(u) and floor(u) + 1,
// zero outside.  Pixel (i, j) sits at (j - c2, i - c1).
//
// The per-ray a, b come from a host table.  Float64 operators evaluate
// u = fma(b, l, a) in float64.  Float32 operators evaluate the same position
// split into an integer and a fraction, in float32 only (GB300's float64 pipe
// is a small fraction of its float32 one): about the middle line l0 of the
// ray, u = ai + af + b (l - l0) with ai an integer and af in [0, 1) (from
// float64 on the host), b = bhi + blo with bhi on a 2^-12 grid, so that
// bhi (l - l0) is exact in float32 for images up to 2048 lines; the integer
// part of bhi (l - l0) is split off exactly and the rest, af + frac + blo
// (l - l0), stays below 3 in magnitude, so the fraction is good to about
// 1e-7.  Either way both kernels evaluate the same expression, so the
// adjoint's interpolation weights are exactly the forward's.
// Forward: one thread per ray, stepping its lines.
// Adjoint: one thread per pixel gathering, angle by angle, the rays whose
// sample on the pixel's row (row-step rays) or column (column-step rays)
// lies within one pixel of it -- bins between those of the rays through the
// points one pixel to either side (the detector coordinate is monotone along
// a line that misses the source), one bin of margin -- each tested with the
// forward's own floor.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace nys {
namespace {

struct FanTab {
    const double* a;       // [n_angles][n_bins]
    const double* b;       // [n_angles][n_bins]
    const double* w;       // [n_angles][n_bins]
    const int* rs;         // [n_angles][n_bins] row-step flag
    const float* ang;      // [n_angles][4]: S_x, S_y, cos, sin
    const float4* split;   // [n_angles][n_bins]: (ai as an integer value, af, bhi, blo) about l0
    float D, du, cb;
    int l0r, l0c;          // middle line of row-step (n1 / 2) and column-step (n2 / 2) rays
};

__device__ __forceinline__ int floor_clamped(double u, double& f) {
    const double fl = floor(fmin(fmax(u, -1.0e9), 1.0e9));
    f = u - fl;
    return (int)fl;
}

// position of ray `ray` on line l: integer part (returned) and fraction f.
// float64 operators: fma(b, l, a) in float64; float32 operators: the split
// float32 evaluation described above.  The forward and the adjoint call this
// same function, so both take the same floor and the same weights.
template <class TC>
__device__ __forceinline__ int fan_pos(const FanTab& tab, int ray, int rs, int l, TC& f);
template <>
__device__ __forceinline__ int fan_pos<double>(const FanTab& tab, int ray, int rs, int l, double& f) {
    return floor_clamped(fma(tab.b[ray], (double)l, tab.a[ray]), f);
}
template <>
__device__ __forceinline__ int fan_pos<float>(const FanTab& tab, int ray, int rs, int l, float& f) {
    const float4 sp = tab.split[ray];
    const float k = (float)(l - (rs ? tab.l0r : tab.l0c));
    const float t = sp.z * k;                 // exact: bhi on a 2^-12 grid, |k| <= 1024
    const float ft = floorf(t);
    const float fr = fmaf(sp.w, k, sp.y + (t - ft));
    const float ff = floorf(fr);
    f = fr - ff;
    const float ip = sp.x + ft + ff;          // an integer below 2^24 in magnitude: exact
    return (int)fminf(fmaxf(ip, -1.0e9f), 1.0e9f);
}

template <class TI, class TO, class TC>
__global__ void __launch_bounds__(256) fan_fwd_kernel(const TI* __restrict__ x, TO* __restrict__ y, int n1, int n2,
                                                      int n_angles, int n_bins, FanTab tab) {
    pdl_enter();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y, b = blockIdx.z;
    if (m >= n_bins) return;
    const int ray = k * n_bins + m;
    const int rs = tab.rs[ray];
    const double a = 0.0, s = 0.0;
    const int nl = rs ? n1 : n2, na = rs ? n2 : n1;
    const TI* xb = x + (size_t)b * n1 * n2;
    TC acc = TC(0);
    (void)a;
    (void)s;
    for (int l = 0; l < nl; ++l) {
        TC f;
        const int lo = fan_pos<TC>(tab, ray, rs, l, f);
        TC v0 = TC(0), v1 = TC(0);
        if ((unsigned)lo < (unsigned)na) v0 = (TC)ldf(xb + (rs ? (size_t)l * n2 + lo : (size_t)lo * n2 + l));
        if ((unsigned)(lo + 1) < (unsigned)na)
            v1 = (TC)ldf(xb + (rs ? (size_t)l * n2 + lo + 1 : (size_t)(lo + 1) * n2 + l));
        acc = fma(TC(1) - f, v0, acc);
        acc = fma(f, v1, acc);
    }
    stf(y + ((size_t)b * n_angles + k) * n_bins + m, (TC)tab.w[ray] * acc);
}

// fractional bin of the ray from the source through (px, py)
__device__ __forceinline__ float fan_bin(const float* g, float px, float py, float D, float du, float cb) {
    const float vx = px - g[0], vy = py - g[1];
    const float along = vx * g[3] * -1.0f + vy * g[2];        // (P - S) . e_d
    const float depth = -(vx * g[2] + vy * g[3]);             // (P - S) . (-e_s)
    return D * along / depth / du + cb;
}

template <class TI, class TO, class TC>
__global__ void __launch_bounds__(256) fan_adj_kernel(const TI* __restrict__ s, TO* __restrict__ x, int n1, int n2,
                                                      int n_angles, int n_bins, FanTab tab) {
    pdl_enter();
    const int64_t N = (int64_t)n1 * n2;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int b = blockIdx.z;
    if (t >= N) return;
    const int i = (int)(t / n2), j = (int)(t - (int64_t)i * n2);
    const float px = (float)j - 0.5f * (float)(n2 - 1), py = (float)i - 0.5f * (float)(n1 - 1);
    const TI* sb = s + (size_t)b * n_angles * n_bins;
    TC acc = TC(0);
    for (int k = 0; k < n_angles; ++k) {
        const float* g = tab.ang + 4 * k;
        // the rays that reach this pixel pass within one pixel of it, so their
        // directions differ from the source-to-pixel direction v by at most
        // asin(1/depth): away from the 45-degree split (|v_y| = |v_x|, where
        // tan changes by 2 per radian) only one kind of ray can reach it
        const float vx = px - g[0], vy = py - g[1];
        const float depth = -(vx * g[2] + vy * g[3]);
        const float tol = 8.0f / depth;
        const bool try_row = fabsf(vy) >= fabsf(vx) * (1.0f - tol);
        const bool try_col = fabsf(vx) >= fabsf(vy) * (1.0f - tol);
        TC part = TC(0);
#pragma unroll
        for (int kind = 0; kind < 2; ++kind) {          // row-step rays (via row i), then column-step (via column j)
            if (!(kind == 0 ? try_row : try_col)) continue;
            const float m1 = kind == 0 ? fan_bin(g, px - 1.0f, py, tab.D, tab.du, tab.cb)
                                       : fan_bin(g, px, py - 1.0f, tab.D, tab.du, tab.cb);
            const float m2 = kind == 0 ? fan_bin(g, px + 1.0f, py, tab.D, tab.du, tab.cb)
                                       : fan_bin(g, px, py + 1.0f, tab.D, tab.du, tab.cb);
            const int mlo = max(0, (int)floorf(fminf(m1, m2)) - 1);
            const int mhi = min(n_bins - 1, (int)ceilf(fmaxf(m1, m2)) + 1);
            const int l = kind == 0 ? i : j, p = kind == 0 ? j : i;
            for (int m = mlo; m <= mhi; ++m) {
                const int ray = k * n_bins + m;
                if (tab.rs[ray] != (kind == 0)) continue;
                TC fd;
                const int lo = fan_pos<TC>(tab, ray, kind == 0, l, fd);
                TC wgt;
                if (lo == p) wgt = TC(1) - fd;
                else if (lo + 1 == p) wgt = fd;
                else continue;
                part = fma((TC)tab.w[ray] * wgt, (TC)ldf(sb + (size_t)ray), part);
            }
        }
        acc += part;
    }
    stf(x + (size_t)b * N + t, acc);
}

// byte offset of the float4 split table in op->rtab: after a, b, w (doubles),
// the row-step flags and the per-angle floats, rounded up to 16 bytes
size_t fan_split_offset(const nys_op* op) {
    const size_t R = (size_t)op->n_angles * op->n_bins;
    const size_t off = 3 * R * sizeof(double) + ((R + 3) & ~size_t(3)) * sizeof(int) +
                       (((size_t)op->n_angles * 4 + 3) & ~size_t(3)) * sizeof(float);
    return (off + 15) & ~size_t(15);
}

FanTab fan_tab(const nys_op* op) {
    const size_t R = (size_t)op->n_angles * op->n_bins;
    const char* base = (const char*)op->rtab;
    FanTab t;
    t.a = (const double*)base;
    t.b = t.a + R;
    t.w = t.b + R;
    t.rs = (const int*)(t.w + R);
    t.ang = (const float*)(t.rs + ((R + 3) & ~size_t(3)));
    t.split = (const float4*)(base + fan_split_offset(op));
    t.l0r = op->n1 / 2;
    t.l0c = op->n2 / 2;
    t.D = (float)op->det_dist;
    t.du = (float)op->det_spacing;
    t.cb = 0.5f * (float)(op->n_bins - 1);
    return t;
}

template <class TI, class TO, class TC>
int fan_fwd(nys_op* op, const void* x, void* y, int batch) {
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int nb = std::min(65535, batch - b0);
        dim3 grid((op->n_bins + 255) / 256, op->n_angles, nb);
        NYS_CK(op->ctx, launch_pdl(fan_fwd_kernel<TI, TO, TC>, grid, 256, 0, op->ctx->stream,
                                   (const TI*)x + (size_t)b0 * op->N, (TO*)y + (size_t)b0 * op->M, op->n1, op->n2,
                                   op->n_angles, op->n_bins, fan_tab(op)));
        NYS_LAUNCH_CK(op->ctx);
    }
    return NYS_OK;
}

template <class TI, class TO, class TC>
int fan_adj(nys_op* op, const void* s, void* x, int batch) {
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int nb = std::min(65535, batch - b0);
        dim3 grid((unsigned)((op->N + 255) / 256), 1, nb);
        NYS_CK(op->ctx, launch_pdl(fan_adj_kernel<TI, TO, TC>, grid, 256, 0, op->ctx->stream,
                                   (const TI*)s + (size_t)b0 * op->M, (TO*)x + (size_t)b0 * op->N, op->n1, op->n2,
                                   op->n_angles, op->n_bins, fan_tab(op)));
        NYS_LAUNCH_CK(op->ctx);
    }
    return NYS_OK;
}

template <class TI, class TO, class TC>
int fan_typed(nys_op* op, int which, const void* x, void* y, int batch) {
    if (which == 0) return fan_fwd<TI, TO, TC>(op, x, y, batch);
    if (which == 1) return fan_adj<TI, TO, TC>(op, x, y, batch);
    for (int b0 = 0; b0 < batch; b0 += op->chunk) {
        const int nb = std::min(op->chunk, batch - b0);
        if (int st = fan_fwd<TI, TC, TC>(op, (const TI*)x + (size_t)b0 * op->N, op->inter, nb)) return st;
        if (int st = fan_adj<TC, TO, TC>(op, op->inter, (TO*)y + (size_t)b0 * op->N, nb)) return st;
    }
    return NYS_OK;
}

}  // namespace

int fanbeam_setup(nys_op* op) {
    const int A = op->n_angles, B = op->n_bins, n1 = op->n1, n2 = op->n2;
    if (op->dtype != NYS_F64 && std::max(n1, n2) > 2048)
        return fail(op->ctx, NYS_EINVAL, "fan beam: float32 operators take images of at most 2048 lines");
    const double c1 = (n1 - 1) / 2.0, c2 = (n2 - 1) / 2.0, cb = (B - 1) / 2.0;
    const double R = op->src_dist, D = op->det_dist, du = op->det_spacing;
    const size_t RA = (size_t)A * B;
    std::vector<double> a(RA), bb(RA), w(RA);
    std::vector<int> rs((RA + 3) & ~size_t(3), 0);
    std::vector<float> ang((size_t)A * 4);
    std::vector<float> split(4 * RA);
    const int l0r = n1 / 2, l0c = n2 / 2;
    for (int k = 0; k < A; ++k) {
        const double th = k * (op->span / A);
        const double cs = std::cos(th), sn = std::sin(th);
        const double Sx = R * cs, Sy = R * sn;
        ang[4 * k] = (float)Sx;
        ang[4 * k + 1] = (float)Sy;
        ang[4 * k + 2] = (float)cs;
        ang[4 * k + 3] = (float)sn;
        for (int m = 0; m < B; ++m) {
            const double um = (m - cb) * du;
            const double dx = -D * cs - um * sn, dy = -D * sn + um * cs;
            const double nd = std::sqrt(dx * dx + dy * dy);
            const bool row = std::fabs(dy) >= std::fabs(dx);
            const size_t r = (size_t)k * B + m;
            const double major = row ? dy : dx, minor = row ? dx : dy;
            bb[r] = minor / major;
            a[r] = row ? Sx - (c1 + Sy) * bb[r] + c2 : Sy - (c2 + Sx) * bb[r] + c1;
            w[r] = nd / std::fabs(major);
            rs[r] = row ? 1 : 0;
            // float32 split about the middle line (see the header comment)
            const double bhi = std::nearbyint(bb[r] * 4096.0) / 4096.0;
            const double am = a[r] + bb[r] * (row ? l0r : l0c);
            const double ai = std::floor(am);
            split[4 * r] = (float)ai;
            split[4 * r + 1] = (float)(am - ai);
            split[4 * r + 2] = (float)bhi;
            split[4 * r + 3] = (float)(bb[r] - bhi);
        }
    }
    const size_t split_off = fan_split_offset(op);
    const size_t bytes = split_off + split.size() * sizeof(float);
    NYS_CK(op->ctx, cudaMalloc(&op->rtab, bytes));
    char* p = (char*)op->rtab;
    NYS_CK(op->ctx, cudaMemcpy(p, a.data(), RA * sizeof(double), cudaMemcpyHostToDevice));
    NYS_CK(op->ctx, cudaMemcpy(p + RA * sizeof(double), bb.data(), RA * sizeof(double), cudaMemcpyHostToDevice));
    NYS_CK(op->ctx, cudaMemcpy(p + 2 * RA * sizeof(double), w.data(), RA * sizeof(double), cudaMemcpyHostToDevice));
    NYS_CK(op->ctx, cudaMemcpy(p + 3 * RA * sizeof(double), rs.data(), rs.size() * sizeof(int),
                               cudaMemcpyHostToDevice));
    NYS_CK(op->ctx, cudaMemcpy(p + 3 * RA * sizeof(double) + rs.size() * sizeof(int), ang.data(),
                               ang.size() * sizeof(float), cudaMemcpyHostToDevice));
    NYS_CK(op->ctx, cudaMemcpy(p + split_off, split.data(), split.size() * sizeof(float), cudaMemcpyHostToDevice));
    op->chunk = 32;
    NYS_CK(op->ctx, cudaMalloc(&op->inter, (size_t)op->chunk * op->M * dtype_size(op->dtype)));
    return NYS_OK;
}

int fanbeam_run(nys_op* op, int which, const void* x, void* y, int batch, int in_dt, int out_dt) {
    if (op->dtype == NYS_F64) {
        if (in_dt != NYS_F64 || out_dt != NYS_F64) return fail(op->ctx, NYS_EINVAL, "f64 operator needs f64 data");
        return fan_typed<double, double, double>(op, which, x, y, batch);
    }
    const bool ib = in_dt == NYS_BF16, ob = out_dt == NYS_BF16;
    if (!ib && !ob) return fan_typed<float, float, float>(op, which, x, y, batch);
    if (ib && ob) return fan_typed<__nv_bfloat16, __nv_bfloat16, float>(op, which, x, y, batch);
    if (ib) return fan_typed<__nv_bfloat16, float, float>(op, which, x, y, batch);
    return fan_typed<float, __nv_bfloat16, float>(op, which, x, y, batch);
}

}  // namespace nys
