// Periodic blur H, its adjoint H^T and the normal operator H^T H (Sec. IV-A),
// plus blur + decimation D H (super-resolution).
//
// Definition (correlation form, periodic boundary, odd kh x kw kernel h):
//     (Hx)[i,j] = sum_{a,b} h[a,b] x[(i + a - ch) mod n1, (j + b - cw) mod n2]
// with ch = (kh-1)/2, cw = (kw-1)/2.  H^T is the same correlation with the
// flipped kernel.  When h is rank one (every Gaussian blur), h = u v^T and
// H = H_col(u) H_row(v), so each apply is two 1-D passes, and
// H^T H = H_col(u * u) H_row(v * v) (autocorrelations of length 2k-1,
// centred at k-1): the normal operator is ONE fused separable pass.
//
// Kernel design (sm_103a): one CTA per TY x TX output tile.  The input tile and
// its periodic halo are staged once in shared memory; the row pass writes an
// intermediate tile to shared memory; the column pass writes the output.  Each
// thread computes 8 consecutive outputs of a row (or column) with a sliding
// register window, so every shared-memory load feeds 8 FMAs and the kernel is
// bound by the FP32 FMA pipe rather than by shared-memory bandwidth.  Row
// pitches are odd so that lanes reading consecutive rows hit distinct banks.
#include "internal.cuh"

#include <cmath>

namespace nys {
namespace {

constexpr int RB = 8;  // register block (outputs per thread along a pass)

// Stage rows x cols input values starting at (r0, c0) (periodic) into a
// shared-memory tile of pitch `pitch`: one warp per row, lanes along the row.
// The wrap is one conditional step when the staged extent fits in the image
// (no integer division per element); small images take the modulo.
template <class TI, class TC>
__device__ __forceinline__ void stage_tile(const TI* __restrict__ xb, int n1, int n2, int r0, int c0, int rows,
                                           int cols, TC* __restrict__ s, int pitch) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const bool step = r0 >= -n1 && r0 + rows <= 2 * n1 && c0 >= -n2 && c0 + cols <= 2 * n2;
    constexpr int MQ = 4;   // rows of up to 128 columns: every load of two rows issued before any store
    if (step && cols <= 32 * MQ) {
        for (int ra = warp; ra < rows; ra += 2 * nw) {
            TC v[2][MQ];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = ra + h * nw;
                int gi = r0 + r;
                gi = gi < 0 ? gi + n1 : (gi >= n1 ? gi - n1 : gi);
                const TI* xr = xb + (size_t)gi * n2;
#pragma unroll
                for (int q = 0; q < MQ; ++q) {
                    const int c = lane + 32 * q;
                    int gj = c0 + c;
                    gj = gj < 0 ? gj + n2 : (gj >= n2 ? gj - n2 : gj);
                    v[h][q] = (r < rows && c < cols) ? (TC)ldf(xr + gj) : TC(0);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = ra + h * nw;
#pragma unroll
                for (int q = 0; q < MQ; ++q) {
                    const int c = lane + 32 * q;
                    if (r < rows && c < cols) s[(size_t)r * pitch + c] = v[h][q];
                }
            }
        }
        return;
    }
    for (int r = warp; r < rows; r += nw) {
        int gi = r0 + r;
        gi = step ? (gi < 0 ? gi + n1 : (gi >= n1 ? gi - n1 : gi)) : pmod(gi, n1);
        const TI* xr = xb + (size_t)gi * n2;
        TC* sr = s + (size_t)r * pitch;
        for (int c = lane; c < cols; c += 32) {
            int gj = c0 + c;
            gj = step ? (gj < 0 ? gj + n2 : (gj >= n2 ? gj - n2 : gj)) : pmod(gj, n2);
            sr[c] = (TC)ldf(xr + gj);
        }
    }
}

__host__ __device__ inline int round8(int x) { return (x + 7) & ~7; }
__host__ __device__ inline int odd_pitch(int x) { return x | 1; }

// Sliding-window 1-D correlation of 8 consecutive outputs:
//   acc[r] += sum_{t < Lp} g[t] * src[(r + t) * stride]
template <class TC>
__device__ __forceinline__ void window8(const TC* __restrict__ src, int stride, const TC* __restrict__ g,
                                        int Lp, TC acc[RB]) {
    TC win[RB], nxt[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) win[r] = src[r * stride];
    for (int t0 = 0; t0 < Lp; t0 += RB) {
#pragma unroll
        for (int r = 0; r < RB; ++r) nxt[r] = src[(t0 + RB + r) * stride];
#pragma unroll
        for (int dt = 0; dt < RB; ++dt) {
            const TC gv = g[t0 + dt];
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const TC v = (r + dt < RB) ? win[r + dt] : nxt[r + dt - RB];
                acc[r] = fma(gv, v, acc[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < RB; ++r) win[r] = nxt[r];
    }
}

// The same window over two independent lines (rows or columns) a and b at
// once: the two lines' values sit in the halves of a float2, so one packed
// FMA (FFMA2, sm_100 and later) does the tap for both, with the same
// rounding as two scalar FMAs; half the FMA instructions of two window8
// calls, and the taps loaded once for both lines.
__device__ __forceinline__ void window8x2(const float* __restrict__ sa, const float* __restrict__ sb, int stride,
                                         const float* __restrict__ g, int Lp, float2 acc[RB]) {
    float2 win[RB], nxt[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) win[r] = make_float2(sa[r * stride], sb[r * stride]);
    for (int t0 = 0; t0 < Lp; t0 += RB) {
#pragma unroll
        for (int r = 0; r < RB; ++r) nxt[r] = make_float2(sa[(t0 + RB + r) * stride], sb[(t0 + RB + r) * stride]);
#pragma unroll
        for (int dt = 0; dt < RB; ++dt) {
            const float gv = g[t0 + dt];
            const float2 g2 = make_float2(gv, gv);
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const float2 v = (r + dt < RB) ? win[r + dt] : nxt[r + dt - RB];
                acc[r] = __ffma2_rn(g2, v, acc[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < RB; ++r) win[r] = nxt[r];
    }
}

template <class TC> struct PairWindow { static constexpr bool on = false; };
template <> struct PairWindow<float> { static constexpr bool on = true; };

// y = H_col(gc) H_row(gr) x, separable periodic correlation.
// taps: gc (Lcp entries, zero padded) followed by gr (Lrp entries).
template <class TI, class TO, class TC, int TY, int TX>
__global__ void __launch_bounds__(256) sepcorr_kernel(const TI* __restrict__ x, TO* __restrict__ y, int n1,
                                                      int n2, const TC* __restrict__ taps, int Lcp, int Lrp,
                                                      int cc, int cr) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC* s_tap = reinterpret_cast<TC*>(smem_raw);
    const int rows = TY + Lcp;          // staged input rows = intermediate rows
    const int wcols = TX + Lrp;         // staged input columns
    const int pin = odd_pitch(wcols);
    const int pmid = odd_pitch(TX);
    TC* s_in = s_tap + Lcp + Lrp;
    TC* s_mid = s_in + (size_t)rows * pin;

    const int i0 = blockIdx.y * TY, j0 = blockIdx.x * TX;
    const size_t img = (size_t)blockIdx.z * n1 * n2;
    const TI* xb = x + img;
    for (int t = threadIdx.x; t < Lcp + Lrp; t += blockDim.x) s_tap[t] = taps[t];
    stage_tile<TI, TC>(xb, n1, n2, i0 - cc, j0 - cr, rows, wcols, s_in, pin);
    __syncthreads();
    // row pass: s_mid[r][c] = sum_b gr[b] s_in[r][c + b]
    const TC* gr = s_tap + Lcp;
    TO* yb = y + img;
    if constexpr (PairWindow<TC>::on) {
        // float32: rows r and r + rows / 2 together (rows = TY + Lcp is even)
        const int hr = rows / 2;
        for (int idx = threadIdx.x; idx < hr * (TX / RB); idx += blockDim.x) {
            const int r = idx % hr, sx = idx / hr;
            float2 acc[RB];
#pragma unroll
            for (int k = 0; k < RB; ++k) acc[k] = make_float2(0.0f, 0.0f);
            window8x2(s_in + r * pin + sx * RB, s_in + (r + hr) * pin + sx * RB, 1, gr, Lrp, acc);
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                s_mid[r * pmid + sx * RB + k] = acc[k].x;
                s_mid[(r + hr) * pmid + sx * RB + k] = acc[k].y;
            }
        }
        __syncthreads();
        // column pass: columns c and c + TX / 2 together
        const int hc = TX / 2;
        for (int idx = threadIdx.x; idx < hc * (TY / RB); idx += blockDim.x) {
            const int c = idx % hc, sy = idx / hc;
            float2 acc[RB];
#pragma unroll
            for (int k = 0; k < RB; ++k) acc[k] = make_float2(0.0f, 0.0f);
            const float* base = s_mid + (sy * RB) * pmid + c;
            window8x2(base, base + hc, pmid, s_tap, Lcp, acc);
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                const int gi = i0 + sy * RB + k;
                if (gi >= n1) continue;
                if (j0 + c < n2) stf(yb + (size_t)gi * n2 + j0 + c, acc[k].x);
                if (j0 + c + hc < n2) stf(yb + (size_t)gi * n2 + j0 + c + hc, acc[k].y);
            }
        }
    } else {
        for (int idx = threadIdx.x; idx < rows * (TX / RB); idx += blockDim.x) {
            const int r = idx % rows, sx = idx / rows;
            TC acc[RB];
#pragma unroll
            for (int k = 0; k < RB; ++k) acc[k] = TC(0);
            window8<TC>(s_in + r * pin + sx * RB, 1, gr, Lrp, acc);
#pragma unroll
            for (int k = 0; k < RB; ++k) s_mid[r * pmid + sx * RB + k] = acc[k];
        }
        __syncthreads();
        // column pass: y[i][c] = sum_a gc[a] s_mid[i + a][c]
        for (int idx = threadIdx.x; idx < TX * (TY / RB); idx += blockDim.x) {
            const int c = idx % TX, sy = idx / TX;
            TC acc[RB];
#pragma unroll
            for (int k = 0; k < RB; ++k) acc[k] = TC(0);
            window8<TC>(s_mid + (sy * RB) * pmid + c, pmid, s_tap, Lcp, acc);
            const int gj = j0 + c;
            if (gj < n2) {
#pragma unroll
                for (int k = 0; k < RB; ++k) {
                    const int gi = i0 + sy * RB + k;
                    if (gi < n1) stf(yb + (size_t)gi * n2 + gj, acc[k]);
                }
            }
        }
    }
}

// General (non-separable) periodic correlation with a kh x kw kernel.
// taps: kh rows of kwp entries (zero padded).
template <class TI, class TO, class TC, int TY, int TX>
__global__ void __launch_bounds__(256) corr2d_kernel(const TI* __restrict__ x, TO* __restrict__ y, int n1,
                                                     int n2, const TC* __restrict__ taps, int kh, int kwp,
                                                     int ch, int cw) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC* s_tap = reinterpret_cast<TC*>(smem_raw);
    const int rows = TY + kh - 1;
    const int wcols = TX + kwp;
    const int pin = odd_pitch(wcols);
    TC* s_in = s_tap + kh * kwp;
    const int i0 = blockIdx.y * TY, j0 = blockIdx.x * TX;
    const size_t img = (size_t)blockIdx.z * n1 * n2;
    const TI* xb = x + img;
    for (int t = threadIdx.x; t < kh * kwp; t += blockDim.x) s_tap[t] = taps[t];
    stage_tile<TI, TC>(xb, n1, n2, i0 - ch, j0 - cw, rows, wcols, s_in, pin);
    __syncthreads();
    TO* yb = y + img;
    for (int idx = threadIdx.x; idx < TY * (TX / RB); idx += blockDim.x) {
        const int r = idx % TY, sx = idx / TY;
        TC acc[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) acc[k] = TC(0);
        for (int a = 0; a < kh; ++a) window8<TC>(s_in + (r + a) * pin + sx * RB, 1, s_tap + a * kwp, kwp, acc);
        const int gi = i0 + r;
        if (gi < n1) {
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                const int gj = j0 + sx * RB + k;
                if (gj < n2) stf(yb + (size_t)gi * n2 + gj, acc[k]);
            }
        }
    }
}

// ---------------------------------------------------- blur + decimate ----
// y[p,q] = sum_{a,b} h[a,b] x[(d p + a - ch) mod n1, (d q + b - cw) mod n2]
template <class TI, class TO, class TC>
__global__ void decim_fwd_kernel(const TI* __restrict__ x, TO* __restrict__ y, int n1, int n2, int d,
                                 const TC* __restrict__ h, int kh, int kw, int batch) {
    pdl_enter();
    const int m1 = n1 / d, m2 = n2 / d;
    const int64_t total = (int64_t)batch * m1 * m2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / ((int64_t)m1 * m2));
        const int rem = (int)(t - (int64_t)b * m1 * m2);
        const int p = rem / m2, q = rem - p * m2;
        const TI* xb = x + (size_t)b * n1 * n2;
        const int ch = (kh - 1) / 2, cw = (kw - 1) / 2;
        TC acc = TC(0);
        for (int a = 0; a < kh; ++a) {
            const int gi = pmod(d * p + a - ch, n1);
            for (int bb = 0; bb < kw; ++bb) {
                const int gj = pmod(d * q + bb - cw, n2);
                acc = fma(h[a * kw + bb], (TC)ldf(xb + (size_t)gi * n2 + gj), acc);
            }
        }
        stf(y + t, acc);
    }
}

// x[i,j] = sum over (a,b) with (i - a + ch) = 0 mod d and (j - b + cw) = 0 mod d of
//          h[a,b] y[((i - a + ch) mod n1)/d, ((j - b + cw) mod n2)/d]
template <class TI, class TO, class TC>
__global__ void decim_adj_kernel(const TI* __restrict__ y, TO* __restrict__ x, int n1, int n2, int d,
                                 const TC* __restrict__ h, int kh, int kw, int batch) {
    pdl_enter();
    const int m1 = n1 / d, m2 = n2 / d;
    const int64_t total = (int64_t)batch * n1 * n2;
    const int ch = (kh - 1) / 2, cw = (kw - 1) / 2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / ((int64_t)n1 * n2));
        const int rem = (int)(t - (int64_t)b * n1 * n2);
        const int i = rem / n2, j = rem - i * n2;
        const TI* yb = y + (size_t)b * m1 * m2;
        TC acc = TC(0);
        for (int a = pmod(i + ch, d); a < kh; a += d) {
            const int zi = pmod(i - a + ch, n1) / d;
            for (int bb = pmod(j + cw, d); bb < kw; bb += d) {
                const int zj = pmod(j - bb + cw, n2) / d;
                acc = fma(h[a * kw + bb], (TC)ldf(yb + (size_t)zi * m2 + zj), acc);
            }
        }
        stf(x + t, acc);
    }
}

// --------------------------------------------------------------- launch --
template <class TC>
size_t sep_smem(int TY, int TX, int Lcp, int Lrp) {
    const int rows = TY + Lcp;
    return sizeof(TC) * ((size_t)(Lcp + Lrp) + (size_t)rows * odd_pitch(TX + Lrp) + (size_t)rows * odd_pitch(TX));
}
template <class TC>
size_t c2d_smem(int TY, int TX, int kh, int kwp) {
    return sizeof(TC) * ((size_t)kh * kwp + (size_t)(TY + kh - 1) * odd_pitch(TX + kwp));
}

template <class TI, class TO, class TC, int T>
int launch_sep(nys_op* op, const void* x, void* y, int batch, const void* taps, int Lcp, int Lrp, int cc,
               int cr) {
    const size_t sm = sep_smem<TC>(T, T, Lcp, Lrp);
    auto k = sepcorr_kernel<TI, TO, TC, T, T>;
    if (sm > 227 * 1024) return fail(op->ctx, NYS_EINVAL, "blur kernel too wide for the shared-memory tile");
    if (int st = smem_optin(op->ctx, (const void*)k, sm)) return st;
    for (int b0 = 0; b0 < batch; b0 += 65535) {     // images in grid.z
        dim3 grid((op->n2 + T - 1) / T, (op->n1 + T - 1) / T, std::min(65535, batch - b0));
        NYS_CK(op->ctx, launch_pdl(k, grid, 256, sm, op->ctx->stream, (const TI*)x + (size_t)b0 * op->N,
                                   (TO*)y + (size_t)b0 * op->N, op->n1, op->n2, (const TC*)taps, Lcp, Lrp, cc, cr));
        NYS_LAUNCH_CK(op->ctx);
    }
    return NYS_OK;
}

template <class TI, class TO, class TC, int T>
int launch_c2d(nys_op* op, const void* x, void* y, int batch, const void* taps) {
    const int kwp = round8(op->kw);
    const size_t sm = c2d_smem<TC>(T, T, op->kh, kwp);
    auto k = corr2d_kernel<TI, TO, TC, T, T>;
    if (sm > 227 * 1024) return fail(op->ctx, NYS_EINVAL, "blur kernel too large for the shared-memory tile");
    if (int st = smem_optin(op->ctx, (const void*)k, sm)) return st;
    for (int b0 = 0; b0 < batch; b0 += 65535) {     // images in grid.z
        dim3 grid((op->n2 + T - 1) / T, (op->n1 + T - 1) / T, std::min(65535, batch - b0));
        NYS_CK(op->ctx, launch_pdl(k, grid, 256, sm, op->ctx->stream, (const TI*)x + (size_t)b0 * op->N,
                                   (TO*)y + (size_t)b0 * op->N, op->n1, op->n2, (const TC*)taps, op->kh, kwp,
                                   (op->kh - 1) / 2, (op->kw - 1) / 2));
        NYS_LAUNCH_CK(op->ctx);
    }
    return NYS_OK;
}

template <class TI, class TO, class TC, int T>
int blur_typed_t(nys_op* op, int which, const void* x, void* y, int batch) {
    if (op->separable) {
        if (which == 2)
            return launch_sep<TI, TO, TC, T>(op, x, y, batch, op->taps_nrm, op->Lc_n, op->Lr_n, op->cc_n, op->cr_n);
        return launch_sep<TI, TO, TC, T>(op, x, y, batch, which == 0 ? op->taps_fwd : op->taps_adj, op->Lc_f,
                                         op->Lr_f, op->cc_f, op->cr_f);
    }
    if (which != 2) return launch_c2d<TI, TO, TC, T>(op, x, y, batch, which == 0 ? op->taps_fwd : op->taps_adj);
    // non-separable normal: H^T (H x) through the intermediate buffer, in chunks
    for (int b0 = 0; b0 < batch; b0 += op->chunk) {
        const int nb = std::min(op->chunk, batch - b0);
        const size_t in_off = (size_t)b0 * op->N * sizeof(TI), out_off = (size_t)b0 * op->N * sizeof(TO);
        if (int st = launch_c2d<TI, TC, TC, T>(op, (const char*)x + in_off, op->inter, nb, op->taps_fwd)) return st;
        if (int st = launch_c2d<TC, TO, TC, T>(op, op->inter, (char*)y + out_off, nb, op->taps_adj)) return st;
    }
    return NYS_OK;
}

// output tile: 32 x 32 in float64; 32 or 64 in float32 (nys_op_autotune picks)
template <class TI, class TO, class TC>
int blur_typed(nys_op* op, int which, const void* x, void* y, int batch) {
    if (sizeof(TC) == 8 || op->blur_tile == 32) return blur_typed_t<TI, TO, TC, 32>(op, which, x, y, batch);
    return blur_typed_t<TI, TO, TC, 64>(op, which, x, y, batch);
}

template <class TI, class TO, class TC>
int decim_typed(nys_op* op, int which, const void* x, void* y, int batch) {
    cudaStream_t s = op->ctx->stream;
    const TC* h = (const TC*)op->taps_fwd;
    const int grid = op->ctx->sm_count * 8;
    if (which == 0) {
        NYS_CK(op->ctx, launch_pdl(decim_fwd_kernel<TI, TO, TC>, grid, 256, 0, s, (const TI*)x, (TO*)y, op->n1,
                                   op->n2, op->decim, h, op->kh, op->kw, batch));
        NYS_LAUNCH_CK(op->ctx);
        return NYS_OK;
    }
    if (which == 1) {
        NYS_CK(op->ctx, launch_pdl(decim_adj_kernel<TI, TO, TC>, grid, 256, 0, s, (const TI*)x, (TO*)y, op->n1,
                                   op->n2, op->decim, h, op->kh, op->kw, batch));
        NYS_LAUNCH_CK(op->ctx);
        return NYS_OK;
    }
    for (int b0 = 0; b0 < batch; b0 += op->chunk) {
        const int nb = std::min(op->chunk, batch - b0);
        NYS_CK(op->ctx, launch_pdl(decim_fwd_kernel<TI, TC, TC>, grid, 256, 0, s, (const TI*)x + (size_t)b0 * op->N,
                                   (TC*)op->inter, op->n1, op->n2, op->decim, h, op->kh, op->kw, nb));
        NYS_LAUNCH_CK(op->ctx);
        NYS_CK(op->ctx, launch_pdl(decim_adj_kernel<TC, TO, TC>, grid, 256, 0, s, (const TC*)op->inter,
                                   (TO*)y + (size_t)b0 * op->N, op->n1, op->n2, op->decim, h, op->kh, op->kw, nb));
        NYS_LAUNCH_CK(op->ctx);
    }
    return NYS_OK;
}

template <template <class, class, class> class F>
struct Dispatch;

// dtype dispatch shared by blur and decimation
template <class Fn>
int dispatch_io(nys_op* op, int in_dt, int out_dt, Fn&& fn) {
    if (op->dtype == NYS_F64) {
        if (in_dt != NYS_F64 || out_dt != NYS_F64) return fail(op->ctx, NYS_EINVAL, "f64 operator needs f64 data");
        return fn((double*)nullptr, (double*)nullptr, (double*)nullptr);
    }
    const bool ib = in_dt == NYS_BF16, ob = out_dt == NYS_BF16;
    if ((in_dt != NYS_F32 && !ib) || (out_dt != NYS_F32 && !ob))
        return fail(op->ctx, NYS_EINVAL, "f32 operator takes f32 or bf16 data");
    if (!ib && !ob) return fn((float*)nullptr, (float*)nullptr, (float*)nullptr);
    if (ib && ob) return fn((__nv_bfloat16*)nullptr, (__nv_bfloat16*)nullptr, (float*)nullptr);
    if (ib) return fn((__nv_bfloat16*)nullptr, (float*)nullptr, (float*)nullptr);
    return fn((float*)nullptr, (__nv_bfloat16*)nullptr, (float*)nullptr);
}

template <class TC>
int upload(nys_op* op, const std::vector<double>& v, void** dst) {
    std::vector<TC> t(v.begin(), v.end());
    NYS_CK(op->ctx, cudaMalloc(dst, t.size() * sizeof(TC) + 16));
    NYS_CK(op->ctx, cudaMemcpy(*dst, t.data(), t.size() * sizeof(TC), cudaMemcpyHostToDevice));
    return NYS_OK;
}

std::vector<double> autocorr(const std::vector<double>& u) {
    const int k = (int)u.size();
    std::vector<double> g(2 * k - 1, 0.0);
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) g[(b - a) + (k - 1)] += u[a] * u[b];
    return g;
}

}  // namespace

int blur_setup(nys_op* op) {
    const int kh = op->kh, kw = op->kw;
    const std::vector<double>& h = op->h;
    // rank-one test: h = u v^T with u = h[:, b*], v = h[a*, :] / h[a*, b*]
    int as = 0, bs = 0;
    double hmax = 0.0;
    for (int a = 0; a < kh; ++a)
        for (int b = 0; b < kw; ++b)
            if (std::fabs(h[a * kw + b]) > hmax) hmax = std::fabs(h[a * kw + b]), as = a, bs = b;
    std::vector<double> u(kh), v(kw);
    for (int a = 0; a < kh; ++a) u[a] = h[a * kw + bs];
    for (int b = 0; b < kw; ++b) v[b] = hmax > 0 ? h[as * kw + b] / h[as * kw + bs] : 0.0;
    double res = 0.0;
    for (int a = 0; a < kh; ++a)
        for (int b = 0; b < kw; ++b) res = std::max(res, std::fabs(h[a * kw + b] - u[a] * v[b]));
    op->separable = hmax > 0 && res <= 1e-13 * hmax;
    const bool f64 = op->dtype == NYS_F64;
    auto up = [&](const std::vector<double>& t, void** dst) {
        return f64 ? upload<double>(op, t, dst) : upload<float>(op, t, dst);
    };
    int st;
    if (op->kind == NYS_OP_BLUR_DECIM) {
        if ((st = up(h, &op->taps_fwd))) return st;
    } else if (op->separable) {
        // forward: [u | v], adjoint: [flip u | flip v]; each padded to a multiple of 8
        op->Lc_f = round8(kh);
        op->Lr_f = round8(kw);
        op->cc_f = (kh - 1) / 2;
        op->cr_f = (kw - 1) / 2;
        std::vector<double> f(op->Lc_f + op->Lr_f, 0.0), g(op->Lc_f + op->Lr_f, 0.0);
        for (int a = 0; a < kh; ++a) f[a] = u[a], g[a] = u[kh - 1 - a];
        for (int b = 0; b < kw; ++b) f[op->Lc_f + b] = v[b], g[op->Lc_f + b] = v[kw - 1 - b];
        if ((st = up(f, &op->taps_fwd))) return st;
        if ((st = up(g, &op->taps_adj))) return st;
        std::vector<double> gu = autocorr(u), gv = autocorr(v);
        op->Lc_n = round8((int)gu.size());
        op->Lr_n = round8((int)gv.size());
        op->cc_n = kh - 1;
        op->cr_n = kw - 1;
        std::vector<double> n(op->Lc_n + op->Lr_n, 0.0);
        for (size_t a = 0; a < gu.size(); ++a) n[a] = gu[a];
        for (size_t b = 0; b < gv.size(); ++b) n[op->Lc_n + b] = gv[b];
        if ((st = up(n, &op->taps_nrm))) return st;
    } else {
        const int kwp = round8(kw);
        std::vector<double> f((size_t)kh * kwp, 0.0), g((size_t)kh * kwp, 0.0);
        for (int a = 0; a < kh; ++a)
            for (int b = 0; b < kw; ++b) {
                f[a * kwp + b] = h[a * kw + b];
                g[a * kwp + b] = h[(kh - 1 - a) * kw + (kw - 1 - b)];
            }
        if ((st = up(f, &op->taps_fwd))) return st;
        if ((st = up(g, &op->taps_adj))) return st;
    }
    // intermediate for two-pass normals: 16 images of the computing type
    const bool twopass = op->kind == NYS_OP_BLUR_DECIM || !op->separable;
    if (twopass) {
        op->chunk = 16;
        NYS_CK(op->ctx, cudaMalloc(&op->inter, (size_t)op->chunk * op->N * (f64 ? 8 : 4)));
    }
    return NYS_OK;
}

int blur_run(nys_op* op, int which, const void* x, void* y, int batch, int in_dt, int out_dt) {
    return dispatch_io(op, in_dt, out_dt, [&](auto* ti, auto* to, auto* tc) {
        using TI = std::remove_pointer_t<decltype(ti)>;
        using TO = std::remove_pointer_t<decltype(to)>;
        using TC = std::remove_pointer_t<decltype(tc)>;
        return blur_typed<TI, TO, TC>(op, which, x, y, batch);
    });
}

int decim_run(nys_op* op, int which, const void* x, void* y, int batch, int in_dt, int out_dt) {
    return dispatch_io(op, in_dt, out_dt, [&](auto* ti, auto* to, auto* tc) {
        using TI = std::remove_pointer_t<decltype(ti)>;
        using TO = std::remove_pointer_t<decltype(to)>;
        using TC = std::remove_pointer_t<decltype(tc)>;
        return decim_typed<TI, TO, TC>(op, which, x, y, batch);
    });
}

}  // namespace nys
