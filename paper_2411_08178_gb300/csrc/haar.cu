// Orthonormal 2-D wavelet transform W (Mallat layout) and W^T, the invertible
// regularisation operator of the wavelet model (Sec. III-B, Eq. with L^{-1}):
// Haar, and Daubechies-4 (the wavelet of the paper's CT experiments) below.
//
// One level on the top-left h x w block maps each 2 x 2 input block
//     [a b; c d] at rows (2p, 2p+1), columns (2q, 2q+1)
// to the four outputs (orthonormal averages / differences)
//     (p, q)          = (a + b + c + d)/2      low-low
//     (p, q + w/2)    = (a - b + c - d)/2      column detail
//     (p + h/2, q)    = (a + b - c - d)/2      row detail
//     (p + h/2, q+w/2)= (a - b - c + d)/2      diagonal detail
// and the next level works on the new h/2 x w/2 low-low block.  One thread
// handles one 2 x 2 block; detail outputs go straight to their final place and
// the low-low block to a ping-pong buffer, so every level is one pass.
#include "internal.cuh"

#include <cmath>

namespace nys {
namespace {

template <class TI, class TO, class TL, class TC>
__global__ void haar_fwd_level(const TI* __restrict__ src, TO* __restrict__ out, TL* __restrict__ ll, int n1,
                               int n2, int h, int w, int last, int batch) {
    pdl_enter();
    const int hh = h / 2, hw = w / 2;
    const int64_t total = (int64_t)batch * hh * hw;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / ((int64_t)hh * hw));
        const int rem = (int)(t - (int64_t)b * hh * hw);
        const int p = rem / hw, q = rem - p * hw;
        const size_t base = (size_t)b * n1 * n2;
        const TI* s = src + base;
        const TC a = ldf(s + (size_t)(2 * p) * n2 + 2 * q), bb = ldf(s + (size_t)(2 * p) * n2 + 2 * q + 1);
        const TC c = ldf(s + (size_t)(2 * p + 1) * n2 + 2 * q), d = ldf(s + (size_t)(2 * p + 1) * n2 + 2 * q + 1);
        const TC half = TC(0.5);
        TO* o = out + base;
        stf(o + (size_t)p * n2 + q + hw, half * ((a - bb) + (c - d)));
        stf(o + (size_t)(p + hh) * n2 + q, half * ((a + bb) - (c + d)));
        stf(o + (size_t)(p + hh) * n2 + q + hw, half * ((a - bb) - (c - d)));
        const TC lo = half * ((a + bb) + (c + d));
        if (last) stf(o + (size_t)p * n2 + q, lo);
        else stf(ll + base + (size_t)p * n2 + q, lo);
    }
}

// inverse level: reads the low-low block from `lsrc` and the three detail
// blocks from `dsrc`, writes the h x w block to `dst`
template <class TL, class TD, class TO, class TC>
__global__ void haar_inv_level(const TL* __restrict__ lsrc, const TD* __restrict__ dsrc, TO* __restrict__ dst,
                               int n1, int n2, int h, int w, int batch) {
    pdl_enter();
    const int hh = h / 2, hw = w / 2;
    const int64_t total = (int64_t)batch * hh * hw;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / ((int64_t)hh * hw));
        const int rem = (int)(t - (int64_t)b * hh * hw);
        const int p = rem / hw, q = rem - p * hw;
        const size_t base = (size_t)b * n1 * n2;
        const TC s0 = ldf(lsrc + base + (size_t)p * n2 + q);
        const TC s1 = ldf(dsrc + base + (size_t)p * n2 + q + hw);
        const TC s2 = ldf(dsrc + base + (size_t)(p + hh) * n2 + q);
        const TC s3 = ldf(dsrc + base + (size_t)(p + hh) * n2 + q + hw);
        const TC half = TC(0.5);
        TO* o = dst + base;
        stf(o + (size_t)(2 * p) * n2 + 2 * q, half * ((s0 + s1) + (s2 + s3)));
        stf(o + (size_t)(2 * p) * n2 + 2 * q + 1, half * ((s0 - s1) + (s2 - s3)));
        stf(o + (size_t)(2 * p + 1) * n2 + 2 * q, half * ((s0 + s1) - (s2 + s3)));
        stf(o + (size_t)(2 * p + 1) * n2 + 2 * q + 1, half * ((s0 - s1) - (s2 - s3)));
    }
}

// ------------------------------------------------------ Daubechies-4 ----
// The periodic four-tap orthonormal filter bank (Daubechies' D4, two
// vanishing moments) in the same layout: along a line of length n,
//     lo[i] = sum_k h[k] x[(2 i + k) mod n],  hi[i] = sum_k g[k] x[(2 i + k) mod n],
// g[k] = (-1)^k h[3 - k], columns first, then rows.  A forward thread reads
// the 4 x 4 input block at rows 2p..2p+3 and columns 2q..2q+3 (modulo the
// current h x w block) and writes the four subband values of (p, q); an
// inverse thread gathers the 2 x 2 coefficient blocks at (p - a, q - b),
// a, b in {0, 1}, of the four subbands for its output pixels 2p..2p+1 x
// 2q..2q+1 (x[2p+r, 2q+c] takes f[r + 2a] f'[c + 2b] times subband (f, f')
// at (p - a, q - b)).
struct D4Taps {
    double h[4], g[4];
};

template <class TI, class TO, class TL, class TC>
__global__ void db4_fwd_level(const TI* __restrict__ src, TO* __restrict__ out, TL* __restrict__ ll, int n1,
                              int n2, int h, int w, int last, int batch, D4Taps f) {
    pdl_enter();
    const int hh = h / 2, hw = w / 2;
    const int64_t total = (int64_t)batch * hh * hw;
    TC fh[4], fg[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) fh[k] = (TC)f.h[k], fg[k] = (TC)f.g[k];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / ((int64_t)hh * hw));
        const int rem = (int)(t - (int64_t)b * hh * hw);
        const int p = rem / hw, q = rem - p * hw;
        const size_t base = (size_t)b * n1 * n2;
        const TI* sb = src + base;
        int jc[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) jc[c] = (2 * q + c) % w;
        TC ll_ = TC(0), lh = TC(0), hl = TC(0), hh_ = TC(0);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const TI* row = sb + (size_t)((2 * p + r) % h) * n2;
            TC lo = TC(0), hi = TC(0);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const TC v = ldf(row + jc[c]);
                lo = fma(fh[c], v, lo);
                hi = fma(fg[c], v, hi);
            }
            ll_ = fma(fh[r], lo, ll_);
            lh = fma(fh[r], hi, lh);
            hl = fma(fg[r], lo, hl);
            hh_ = fma(fg[r], hi, hh_);
        }
        TO* o = out + base;
        stf(o + (size_t)p * n2 + q + hw, lh);
        stf(o + (size_t)(p + hh) * n2 + q, hl);
        stf(o + (size_t)(p + hh) * n2 + q + hw, hh_);
        if (last) stf(o + (size_t)p * n2 + q, ll_);
        else stf(ll + base + (size_t)p * n2 + q, ll_);
    }
}

template <class TL, class TD, class TO, class TC>
__global__ void db4_inv_level(const TL* __restrict__ lsrc, const TD* __restrict__ dsrc, TO* __restrict__ dst,
                              int n1, int n2, int h, int w, int batch, D4Taps f) {
    pdl_enter();
    const int hh = h / 2, hw = w / 2;
    const int64_t total = (int64_t)batch * hh * hw;
    TC fh[4], fg[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) fh[k] = (TC)f.h[k], fg[k] = (TC)f.g[k];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / ((int64_t)hh * hw));
        const int rem = (int)(t - (int64_t)b * hh * hw);
        const int p = rem / hw, q = rem - p * hw;
        const size_t base = (size_t)b * n1 * n2;
        // coefficients of the four subbands at (p - a, q - b)
        TC LL[2][2], LH[2][2], HL[2][2], HH[2][2];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int pa = (p - a + hh) % hh;
#pragma unroll
            for (int bb = 0; bb < 2; ++bb) {
                const int qb = (q - bb + hw) % hw;
                LL[a][bb] = ldf(lsrc + base + (size_t)pa * n2 + qb);
                LH[a][bb] = ldf(dsrc + base + (size_t)pa * n2 + qb + hw);
                HL[a][bb] = ldf(dsrc + base + (size_t)(pa + hh) * n2 + qb);
                HH[a][bb] = ldf(dsrc + base + (size_t)(pa + hh) * n2 + qb + hw);
            }
        }
        TO* o = dst + base;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                TC v = TC(0);
#pragma unroll
                for (int a = 0; a < 2; ++a) {
#pragma unroll
                    for (int bb = 0; bb < 2; ++bb) {
                        const TC hr = fh[r + 2 * a], gr = fg[r + 2 * a], hc = fh[c + 2 * bb], gc = fg[c + 2 * bb];
                        v = fma(hr * hc, LL[a][bb], v);
                        v = fma(hr * gc, LH[a][bb], v);
                        v = fma(gr * hc, HL[a][bb], v);
                        v = fma(gr * gc, HH[a][bb], v);
                    }
                }
                stf(o + (size_t)(2 * p + r) * n2 + 2 * q + c, v);
            }
        }
    }
}

D4Taps db4_taps() {
    const double s3 = std::sqrt(3.0), d = 4.0 * std::sqrt(2.0);
    D4Taps f;
    f.h[0] = (1.0 + s3) / d;
    f.h[1] = (3.0 + s3) / d;
    f.h[2] = (3.0 - s3) / d;
    f.h[3] = (1.0 - s3) / d;
    for (int k = 0; k < 4; ++k) f.g[k] = (k % 2 ? -1.0 : 1.0) * f.h[3 - k];
    return f;
}

// copy the part of the image outside the top-left h x w block (inverse needs
// the finer details copied through; forward writes them directly)
template <class TS, class TD>
__global__ void copy_outside(const TS* __restrict__ src, TD* __restrict__ dst, int n1, int n2, int h, int w,
                             int batch) {
    const int64_t total = (int64_t)batch * n1 * n2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int rem = (int)(t % ((int64_t)n1 * n2));
        const int i = rem / n2, j = rem - i * n2;
        if (i >= h || j >= w) stf(dst + t, ldf(src + t));
    }
}

template <class TI, class TO, class TC>
int haar_typed(nys_op* op, const void* in, void* out, int batch, int inverse) {
    nys_ctx* ctx = op->ctx;
    const int n1 = op->n1, n2 = op->n2, L = op->haar_levels;
    const size_t imgs = (size_t)batch * op->N;
    int st;
    TC* tmp = (TC*)scratch(ctx, SLOT_OPTMP, 2 * imgs * sizeof(TC), &st);
    if (st) return st;
    TC* tA = tmp;
    TC* tB = tmp + imgs;
    const int grid = ctx->sm_count * 8;
    cudaStream_t s = ctx->stream;
    if (L == 0) return fail(ctx, NYS_EINVAL, "haar with zero levels");
    const bool db4 = op->wavelet == NYS_WAVELET_DB4;
    const D4Taps taps = db4_taps();
    if (!inverse) {
        const void* src = in;
        bool src_is_in = true;
        TC* cur = tA;
        for (int lev = 0; lev < L; ++lev) {
            const int h = n1 >> lev, w = n2 >> lev, last = (lev == L - 1);
            if (db4 && src_is_in)
                NYS_CK(ctx, launch_pdl(db4_fwd_level<TI, TO, TC, TC>, grid, 256, 0, s,
                                       (const TI*)src, (TO*)out, cur, n1, n2, h, w, last, batch, taps));
            else if (db4)
                NYS_CK(ctx, launch_pdl(db4_fwd_level<TC, TO, TC, TC>, grid, 256, 0, s,
                                       (const TC*)src, (TO*)out, cur, n1, n2, h, w, last, batch, taps));
            else if (src_is_in)
                NYS_CK(ctx, launch_pdl(haar_fwd_level<TI, TO, TC, TC>, grid, 256, 0, s,
                                       (const TI*)src, (TO*)out, cur, n1, n2, h, w, last, batch));
            else
                NYS_CK(ctx, launch_pdl(haar_fwd_level<TC, TO, TC, TC>, grid, 256, 0, s,
                                       (const TC*)src, (TO*)out, cur, n1, n2, h, w, last, batch));
            NYS_LAUNCH_CK(ctx);
            src = cur;
            src_is_in = false;
            cur = (cur == tA) ? tB : tA;
        }
        return NYS_OK;
    }
    // inverse: coarsest level first; low-low comes from `in` at the coarsest
    // level, then from the previous level's result
    const TC* lsrc = nullptr;
    TC* cur = tA;
    for (int lev = L - 1; lev >= 0; --lev) {
        const int h = n1 >> lev, w = n2 >> lev;
        if (lev == 0) {
            if (lev == L - 1 && db4)
                NYS_CK(ctx, launch_pdl(db4_inv_level<TI, TI, TO, TC>, grid, 256, 0, s,
                                       (const TI*)in, (const TI*)in, (TO*)out, n1, n2, h, w, batch, taps));
            else if (db4)
                NYS_CK(ctx, launch_pdl(db4_inv_level<TC, TI, TO, TC>, grid, 256, 0, s,
                                       lsrc, (const TI*)in, (TO*)out, n1, n2, h, w, batch, taps));
            else if (lev == L - 1)
                NYS_CK(ctx, launch_pdl(haar_inv_level<TI, TI, TO, TC>, grid, 256, 0, s,
                                       (const TI*)in, (const TI*)in, (TO*)out, n1, n2, h, w, batch));
            else
                NYS_CK(ctx, launch_pdl(haar_inv_level<TC, TI, TO, TC>, grid, 256, 0, s,
                                       lsrc, (const TI*)in, (TO*)out, n1, n2, h, w, batch));
            NYS_LAUNCH_CK(ctx);
        } else {
            if (lev == L - 1 && db4)
                NYS_CK(ctx, launch_pdl(db4_inv_level<TI, TI, TC, TC>, grid, 256, 0, s,
                                       (const TI*)in, (const TI*)in, cur, n1, n2, h, w, batch, taps));
            else if (db4)
                NYS_CK(ctx, launch_pdl(db4_inv_level<TC, TI, TC, TC>, grid, 256, 0, s,
                                       lsrc, (const TI*)in, cur, n1, n2, h, w, batch, taps));
            else if (lev == L - 1)
                NYS_CK(ctx, launch_pdl(haar_inv_level<TI, TI, TC, TC>, grid, 256, 0, s,
                                       (const TI*)in, (const TI*)in, cur, n1, n2, h, w, batch));
            else
                NYS_CK(ctx, launch_pdl(haar_inv_level<TC, TI, TC, TC>, grid, 256, 0, s,
                                       lsrc, (const TI*)in, cur, n1, n2, h, w, batch));
            NYS_LAUNCH_CK(ctx);
            lsrc = cur;
            cur = (cur == tA) ? tB : tA;
        }
    }
    (void)copy_outside<TI, TO>;
    return NYS_OK;
}

}  // namespace

int haar_run(nys_op* op, const void* in, void* out, int batch, int inverse, int in_dt, int out_dt) {
    if (op->dtype == NYS_F64) {
        if (in_dt != NYS_F64 || out_dt != NYS_F64) return fail(op->ctx, NYS_EINVAL, "haar: f64 data expected");
        return haar_typed<double, double, double>(op, in, out, batch, inverse);
    }
    if (in_dt == NYS_F32 && out_dt == NYS_F32) return haar_typed<float, float, float>(op, in, out, batch, inverse);
    if (in_dt == NYS_BF16 && out_dt == NYS_F32) return haar_typed<__nv_bfloat16, float, float>(op, in, out, batch, inverse);
    if (in_dt == NYS_F32 && out_dt == NYS_BF16) return haar_typed<float, __nv_bfloat16, float>(op, in, out, batch, inverse);
    if (in_dt == NYS_BF16 && out_dt == NYS_BF16)
        return haar_typed<__nv_bfloat16, __nv_bfloat16, float>(op, in, out, batch, inverse);
    return fail(op->ctx, NYS_EINVAL, "haar: unsupported dtypes");
}

}  // namespace nys
