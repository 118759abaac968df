// Orthonormal 2-D Haar transform W (Mallat layout) and W^T, the invertible
// regularisation operator of the wavelet model (Sec. III-B, Eq. with L^{-1}).
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
    if (!inverse) {
        const void* src = in;
        bool src_is_in = true;
        TC* cur = tA;
        for (int lev = 0; lev < L; ++lev) {
            const int h = n1 >> lev, w = n2 >> lev, last = (lev == L - 1);
            if (src_is_in)
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
            if (lev == L - 1)
                NYS_CK(ctx, launch_pdl(haar_inv_level<TI, TI, TO, TC>, grid, 256, 0, s,
                                       (const TI*)in, (const TI*)in, (TO*)out, n1, n2, h, w, batch));
            else
                NYS_CK(ctx, launch_pdl(haar_inv_level<TC, TI, TO, TC>, grid, 256, 0, s,
                                       lsrc, (const TI*)in, (TO*)out, n1, n2, h, w, batch));
            NYS_LAUNCH_CK(ctx);
        } else {
            if (lev == L - 1)
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
