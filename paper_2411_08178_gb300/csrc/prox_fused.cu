// Dual APG step of the P-metric prox (Sec. III-B) for a low-rank
// preconditioner P = I + Ubar Ubar^T, P^{-1} z = z - U M U^T z over the active
// columns of U (Eq. RYPreconditioner in Woodbury form).  One dual step
//     x   = s - lb P^{-1} L^T R
//     Q'  = Proj(R + step L x),  R <- Q' + beta (Q' - Q),  Q <- Q'
// takes two launches for anisotropic TV (three for HS) instead of six:
//   lt_utz   TV: the dual update of the previous step fused in front of
//            g = L^T R_new (stencil.cuh, tv_dual_lt; HS: g = L^T R) over a
//            chunk of pixels, written out and staged in shared memory, then
//            the chunk's partial sums of U^T g (warps over the active
//            columns, 16-byte loads of U); the last CTA to finish reduces the
//            (column-major) partials and forms c = M w
//   uc       x = s - lb (g - U c)   (vec.cuh, 16-byte loads of U)
//   dual     HS only: L x and the dual update (stencil.cuh)
// U is read twice per step, as in the unfused P^{-1} apply; the launches of
// L^T R, the coefficient pass and x = s - lb (...) are folded away.
#include "internal.cuh"
#include "stencil.cuh"
#include "vec.cuh"

#include <algorithm>
#include <cmath>

namespace nys {
namespace {

constexpr int FCH = 1024;        // pixels per partial-sum chunk (small active sets)
constexpr int FCH_WIDE = 512;    // large active sets: twice the CTAs, more bytes of U in flight
constexpr int COUNTER_PROX = 1;

// The x of the previous dual step, x = s - lb (g - U c), for a step that
// stages it in shared memory instead of reading a stored x (c: le <= 64)
template <class T, class TA>
struct XStage {
    const T* s;
    const T* g;
    const TA* c;
    TA lb;
};

// DUAL: the stencil pass is the anisotropic-TV dual step fused with the L^T
// after it (tv_dual_lt, inputs and outputs in `dual`, R unused); otherwise
// it is L^T R.  XR (with DUAL, small active sets): the CTA first computes x
// on its chunk and one image row either side (U c from 16-byte loads of the
// L2-resident U, one chain of FMAs over the columns per pixel, so a pixel
// staged by two CTAs gets the same float in both) into shared memory, and
// the stencil reads it there: one launch per dual step, no stored x.
// Dynamic shared memory: XR: FCH + 2 n2 + 64 values, then the last CTA's.
template <class TU, class T, class TA, class TM, int REG, bool LAST, int FCH, bool DUAL, bool XR = false>
__global__ void __launch_bounds__(256) lt_utz_kernel(const T* __restrict__ R, int n1, int n2,
                                                     const TU* __restrict__ U, int le, int ldm,
                                                     const TM* __restrict__ M, T* __restrict__ g,
                                                     TA* __restrict__ part, TA* __restrict__ coef,
                                                     unsigned* __restrict__ counter, TvDual<T> dual, int keep,
                                                     XStage<T, TA> xr, DualStop stop) {
    pdl_enter();
    static_assert(!DUAL || REG == NYS_REG_TV, "the fused dual step is for anisotropic TV");
    static_assert(!XR || DUAL, "x is staged only for the fused dual step");
    constexpr int V = Vec16<TU>::n;
    constexpr int PT = (FCH + 255) / 256;   // pixels per thread in the stencil pass
    __shared__ __align__(16) TA gs[FCH];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t N = (int64_t)n1 * n2;
    const int64_t i0 = (int64_t)blockIdx.x * FCH;
    const int nst = XR ? FCH + 2 * n2 : 0;          // staged x values
    TA* xs = reinterpret_cast<TA*>(smem_raw);
    TA* cs = xs + nst;
    TA* sm = XR ? cs + 64 : xs;   // last CTA: w and (le <= 64) M
    const int64_t base = XR ? (i0 - n2 + N) % N : 0;   // first staged pixel
    if constexpr (DUAL) {
        // the exact early stop (internal.cuh): a skipped step writes nothing
        // (the last one only Q)
        const bool skip = dual_skip(stop);
        dual_stop_enter(stop, skip);
        if (skip) {
            if (!dual.Rn)
                for (int q = threadIdx.x; q < FCH && i0 + q < N; q += blockDim.x)
                    tv_dual_copy_q<T>(dual, (size_t)(i0 + q), (size_t)N);
            return;
        }
    } else {
        // L^T R of an unfused dual step (the dual update keeps the flags)
        if (dual_skip(stop)) return;
    }
    if constexpr (XR) {
        for (int k = threadIdx.x; k < le; k += blockDim.x) cs[k] = xr.c[k];
        __syncthreads();
        // V consecutive pixels per thread and round (base, N and n2 are
        // multiples of V, so a vector never wraps)
        for (int v0 = threadIdx.x * V; v0 < nst; v0 += blockDim.x * V) {
            const int64_t q0 = (base + v0) % N;
            TA acc[V];
#pragma unroll
            for (int e = 0; e < V; ++e) acc[e] = TA(0);
            for (int k = 0; k < le; ++k) {
                TA u[V];
                load_vec<TU, TA, V>(U + (size_t)k * N + q0, u);
                const TA ck = cs[k];
#pragma unroll
                for (int e = 0; e < V; ++e) acc[e] = fma(u[e], ck, acc[e]);
            }
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const TA v = (TA)xr.g[q0 + e] + TA(-1) * acc[e];
                xs[v0 + e] = (TA)xr.s[q0 + e] + (-xr.lb) * v;
            }
        }
        __syncthreads();
    }
    using TC = typename Comp<T>::type;
    auto xf = [&](size_t q) -> TC {
        int64_t o = (int64_t)q - base;
        if (o < 0) o += N;
        return (TC)xs[o];
    };
    TA v[PT];
    bool chg = false;
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const int64_t p = i0 + threadIdx.x + q * 256;
        v[q] = TA(0);
        if (threadIdx.x + q * 256 < FCH && p < N) {
            int i, j;
            pix_ij(p, n2, i, j);
            if constexpr (XR)
                v[q] = (TA)tv_dual_lt_f<T>(dual, xf, i, j, n1, n2, &chg);
            else
                v[q] = DUAL ? (TA)tv_dual_lt<T>(dual, i, j, n1, n2, &chg) : (TA)lt_q<T, REG>(R, i, j, n1, n2);
        }
    }
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const int64_t p = i0 + threadIdx.x + q * 256;
        if (threadIdx.x + q * 256 >= FCH) continue;
        if (p < N) g[p] = (T)v[q];
        gs[threadIdx.x + q * 256] = v[q];
    }
    if constexpr (DUAL) dual_stop_report(stop, chg);   // (a block barrier)
    else __syncthreads();
    if (le == 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cnt = (int)(N - i0 < (int64_t)FCH ? N - i0 : (int64_t)FCH);   // multiple of V
    constexpr int T4 = FCH / (32 * V);
    const L2Pol l2p = make_l2_pol();
    for (int j = warp; j < le; j += 16) {
        // columns j and j + 8 together: twice the 16-byte loads in flight
        const bool two = j + 8 < le;
        const TU* u0 = U + (size_t)j * N + i0;
        const TU* u1 = U + (size_t)(two ? j + 8 : j) * N + i0;
        const uint64_t p0 = j < keep ? l2p.last : l2p.first;
        const uint64_t p1 = (two ? j + 8 : j) < keep ? l2p.last : l2p.first;
        TA s0 = TA(0), s1 = TA(0);
        if (cnt == FCH) {
            TA a[T4][V], b[T4][V];
#pragma unroll
            for (int q = 0; q < T4; ++q) {
                load_vec_pol<TU, TA, V>(u0 + (q * 32 + lane) * V, a[q], p0);
                load_vec_pol<TU, TA, V>(u1 + (q * 32 + lane) * V, b[q], p1);
            }
#pragma unroll
            for (int q = 0; q < T4; ++q) {
                TA zv[V];
                lds_vec<TA, V>(gs + (q * 32 + lane) * V, zv);
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    s0 = fma(a[q][k], zv[k], s0);
                    s1 = fma(b[q][k], zv[k], s1);
                }
            }
        } else {
            for (int t = lane * V; t < cnt; t += 32 * V) {
                TA a[V], b[V], zv[V];
                load_vec_pol<TU, TA, V>(u0 + t, a, p0);
                load_vec_pol<TU, TA, V>(u1 + t, b, p1);
                lds_vec<TA, V>(gs + t, zv);
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    s0 = fma(a[k], zv[k], s0);
                    s1 = fma(b[k], zv[k], s1);
                }
            }
        }
        s0 = warp_sum(s0);
        s1 = warp_sum(s1);
        if (lane == 0) {
            part[(size_t)j * gridDim.x + blockIdx.x] = s0;
            if (two) part[(size_t)(j + 8) * gridDim.x + blockIdx.x] = s1;
        }
    }
    if (LAST) last_cta_coef_t<TA, TM>(part, le, ldm, M, coef, counter, sm);
}

template <class TU, class T, class TA, int REG>
int fused_typed(nys_ctx* ctx, const nys_precond* pc, double lb, int n_inner, int n1, int n2, const T* s, T* out,
                T* Q) {
    using TM = typename std::conditional<sizeof(TA) == 8, double, float>::type;
    constexpr int V = Vec16<TU>::n;
    constexpr bool TV = REG == NYS_REG_TV;
    const nys_precond_priv* pv = (const nys_precond_priv*)pc->priv;
    const int G = dual_components(REG);
    const double normL2 = first_order(REG) ? 8.0 : 32.0;
    const int64_t N = (int64_t)n1 * n2;
    const int le = pv->ell_eff;
    // small active sets: the last CTA of lt_utz forms M w; large ones: two
    // passes over many CTAs (reduce_cols, mw) and smaller pixel chunks (more
    // CTAs, more bytes of U in flight)
    const bool last = le <= 64;
    const int fch = last ? FCH : FCH_WIDE;
    const int nchunk = (int)((N + fch - 1) / fch);
    int st;
    T* work = (T*)scratch(ctx, SLOT_PROX, prox_work_elems(G, N) * sizeof(T), &st);
    if (st) return st;
    T* g = work;
    T* x = g + N;
    T* RQ[2][2] = {{x + N, x + N + G * N}, {x + N + 2 * G * N, x + N + 3 * G * N}};   // [buffer][R, Q]
    TA* part = (TA*)scratch(ctx, SLOT_PRECOND, ((size_t)nchunk * std::max(le, 1) + 2 * std::max(le, 1)) * sizeof(TA), &st);
    if (st) return st;
    TA* coef = part + (size_t)nchunk * std::max(le, 1);
    TA* wbuf = coef + std::max(le, 1);
    cudaStream_t sm = ctx->stream;
    const TM* M = sizeof(TA) == 8 ? (const TM*)pv->M64 : (const TM*)pv->M32;
    const size_t lsm = ((size_t)le + (le <= 64 ? (size_t)le * le : 0)) * sizeof(TA) + 16;
    // x pass: large active sets take two 16-byte vectors per lane and two
    // columns per round (1 KB contiguous per column and warp)
    const int pvx = last ? 1 : 2;
    const int P = 32 * V * pvx;
    const size_t usm = (((size_t)le + 3) & ~size_t(3)) * sizeof(TA) + (size_t)8 * P * sizeof(TA);
    const int ug = (int)((N + P - 1) / P);
    const int dg = (int)std::min<int64_t>((N + 255) / 256, (int64_t)ctx->sm_count * 8);
    const TA step = (TA)(1.0 / (lb * normL2));
    unsigned* counter = ctx->counters + COUNTER_PROX;
    const int keep = l2_keep_cols(ctx, N, sizeof(TU), le);
    const XStage<T, TA> xr0 = {};
    const DualStop nostop{};
    // the exact early stop of the TV dual iteration for step k (internal.cuh)
    auto stop_at = [&](int k) {
        DualStop ds;
        if (ctx->dual_stop) ds.flags = ctx->counters + COUNTER_DUAL_STOP;
        ds.k = k;
        return ds;
    };
    // g = L^T Rin, or the fused TV dual step and the L^T after it (dual.x
    // set); then x (or out) = s - lb (g - U c), c = M U^T g.  ds: the dual
    // step's early stop (the x pass of the last step always runs)
    auto xfn = [&](const T* Rin, const TvDual<T>& dual, T* dst, DualStop ds) -> int {
        // the last dual step's x pass: if that step is skipped, x already holds
        // its output (the last step that ran computed it from the same g and
        // c; at the fixed point the two L^T agree bit for bit)
        DualStop ucs = ds;
        if (dual.x && !dual.Rn) ucs.copy = dual.x;
        if (last) {
            if (dual.x)
                NYS_CK(ctx, launch_pdl(lt_utz_kernel<TU, T, TA, TM, REG, true, FCH, TV>, nchunk, 256, lsm, sm, Rin,
                                       n1, n2, (const TU*)pc->U, le, pc->ell, M, g, part, coef, counter, dual, keep, xr0, ds));
            else
                NYS_CK(ctx, launch_pdl(lt_utz_kernel<TU, T, TA, TM, REG, true, FCH, false>, nchunk, 256, lsm, sm, Rin,
                                       n1, n2, (const TU*)pc->U, le, pc->ell, M, g, part, coef, counter, dual, keep, xr0, ds));
            NYS_LAUNCH_CK(ctx);
        } else {
            if (dual.x)
                NYS_CK(ctx, launch_pdl(lt_utz_kernel<TU, T, TA, TM, REG, false, FCH_WIDE, TV>, nchunk, 256, 16, sm,
                                       Rin, n1, n2, (const TU*)pc->U, le, pc->ell, M, g, part, coef, counter, dual, keep, xr0, ds));
            else
                NYS_CK(ctx, launch_pdl(lt_utz_kernel<TU, T, TA, TM, REG, false, FCH_WIDE, false>, nchunk, 256, 16, sm,
                                       Rin, n1, n2, (const TU*)pc->U, le, pc->ell, M, g, part, coef, counter, dual, keep, xr0, ds));
            NYS_LAUNCH_CK(ctx);
            int st2 = coef_run<TA, TM>(ctx, part, nchunk, le, pc->ell, 1, M, (const TM*)nullptr, coef, 1, wbuf, ds);
            if (st2) return st2;
        }
        if (pvx == 1)
            NYS_CK(ctx, launch_pdl(uc_vec_kernel<TU, T, TA>, dim3(ug, 1), 256, usm, sm, (const TU*)pc->U, g, N, le,
                                   coef, TA(-1), dst, s, (TA)(-lb), keep, ucs));
        else
            NYS_CK(ctx, launch_pdl(uc_vec_kernel<TU, T, TA, 2, 2>, dim3(ug, 1), 256, usm, sm, (const TU*)pc->U, g, N,
                                   le, coef, TA(-1), dst, s, (TA)(-lb), keep, ucs));
        NYS_LAUNCH_CK(ctx);
        return NYS_OK;
    };
    const TvDual<T> none = {};
    double t = 1.0;
    const size_t xsm = ((size_t)FCH + 2 * (size_t)n2 + 64) * sizeof(TA) + lsm;
    // (48 KB: static gs[FCH] plus this dynamic part, no opt-in needed)
    if (TV && last && n_inner >= 1 && n2 % V == 0 && N >= (int64_t)FCH + 2 * n2 &&
        xsm + (size_t)FCH * sizeof(TA) <= 48 * 1024) {
        // small active sets: one launch per dual step, x staged per chunk from
        // U (L2-resident), c, s and g (XR above); g and c alternate between
        // two buffers; the final x is one pass of U c
        T* gb[2] = {g, x};
        TA* cb[2] = {coef, wbuf};
        NYS_CK(ctx, launch_pdl(lt_utz_kernel<TU, T, TA, TM, REG, true, FCH, false>, nchunk, 256, lsm, sm, Q, n1, n2,
                               (const TU*)pc->U, le, pc->ell, M, gb[0], part, cb[0], counter, none, keep, xr0,
                               nostop));
        NYS_LAUNCH_CK(ctx);
        for (int k = 0; k < n_inner; ++k) {
            const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
            const double beta = (t - 1.0) / tn;
            t = tn;
            const bool fin = k + 1 == n_inner;
            TvDual<T> d;
            d.x = nullptr;
            d.Ro = k ? RQ[k & 1][0] : Q;
            d.Qo = k ? RQ[k & 1][1] : Q;
            d.Rn = fin ? nullptr : RQ[(k + 1) & 1][0];
            d.Qn = (fin && k) ? Q : RQ[(k + 1) & 1][1];
            d.step = step;
            d.beta = (TA)beta;
            const XStage<T, TA> xr = {s, gb[k & 1], cb[k & 1], (TA)lb};
            NYS_CK(ctx, launch_pdl(lt_utz_kernel<TU, T, TA, TM, REG, true, FCH, TV, TV>, nchunk, 256, xsm, sm,
                                   (const T*)nullptr, n1, n2, (const TU*)pc->U, le, pc->ell, M, gb[(k + 1) & 1], part,
                                   cb[(k + 1) & 1], counter, d, keep, xr, stop_at(k)));
            NYS_LAUNCH_CK(ctx);
        }
        NYS_CK(ctx, launch_pdl(uc_vec_kernel<TU, T, TA>, dim3(ug, 1), 256, usm, sm, (const TU*)pc->U, gb[n_inner & 1],
                               N, le, cb[n_inner & 1], TA(-1), out, s, (TA)(-lb), keep, nostop));
        NYS_LAUNCH_CK(ctx);
        if (n_inner == 1) NYS_CK(ctx, cudaMemcpyAsync(Q, RQ[1][1], sizeof(T) * G * N, cudaMemcpyDeviceToDevice, sm));
        return NYS_OK;
    }
    if (TV) {
        // warm start R = Q = Q_in; step k reads (R, Q) from RQ[k & 1] (Q_in
        // itself for k = 0) and writes RQ[(k + 1) & 1]; the last step writes
        // only Q, straight into Q_in when that is not its own input
        if ((st = xfn(Q, none, n_inner ? x : out, nostop))) return st;
        for (int k = 0; k < n_inner; ++k) {
            const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
            const double beta = (t - 1.0) / tn;
            t = tn;
            const bool fin = k + 1 == n_inner;
            TvDual<T> d;
            d.x = x;
            d.Ro = k ? RQ[k & 1][0] : Q;
            d.Qo = k ? RQ[k & 1][1] : Q;
            d.Rn = fin ? nullptr : RQ[(k + 1) & 1][0];
            d.Qn = (fin && k) ? Q : RQ[(k + 1) & 1][1];
            d.step = step;
            d.beta = (TA)beta;
            if ((st = xfn(nullptr, d, fin ? out : x, stop_at(k)))) return st;
        }
        if (n_inner == 1) NYS_CK(ctx, cudaMemcpyAsync(Q, RQ[1][1], sizeof(T) * G * N, cudaMemcpyDeviceToDevice, sm));
        return NYS_OK;
    }
    T* R = RQ[0][0];
    T* Qp = RQ[0][1];
    NYS_CK(ctx, cudaMemcpyAsync(R, Q, sizeof(T) * G * N, cudaMemcpyDeviceToDevice, sm));
    NYS_CK(ctx, cudaMemcpyAsync(Qp, Q, sizeof(T) * G * N, cudaMemcpyDeviceToDevice, sm));
    for (int k = 0; k < n_inner; ++k) {
        // the exact early stop: the dual update keeps the flags, the x pass
        // of a skipped step does nothing (x, R and Q already hold the fixed
        // point)
        if ((st = xfn(R, none, x, stop_at(k)))) return st;
        const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        const double beta = (t - 1.0) / tn;
        t = tn;
        NYS_CK(ctx, launch_pdl(dual_update_kernel<T, REG>, dg, 256, 0, sm, x, R, Qp, step, (TA)beta, n1, n2,
                               stop_at(k)));
        NYS_LAUNCH_CK(ctx);
    }
    NYS_CK(ctx, cudaMemcpyAsync(Q, Qp, sizeof(T) * G * N, cudaMemcpyDeviceToDevice, sm));
    return xfn(Qp, none, out, nostop);
}

}  // namespace

// fused prox for a set-up low-rank P; NYS_EINVAL (nothing launched) when the
// layout does not allow it, so the caller can take the unfused path
int prox_dual_fused(nys_ctx* ctx, const nys_precond* pc, int reg, double lb, int n_inner, int dtype, int n1, int n2,
                    const void* s, void* out, void* Q) {
    if (!pc || !pc->priv) return NYS_EINVAL;
    const nys_precond_priv* pv = (const nys_precond_priv*)pc->priv;
    const int64_t N = (int64_t)n1 * n2;
    const int V = pc->dtype == NYS_BF16 ? 8 : (pc->dtype == NYS_F32 ? 4 : 2);
    const bool aligned = (((uintptr_t)pc->U | (uintptr_t)s | (uintptr_t)out) & 15) == 0;
    if (N % V || N % 4 || !aligned || pv->ell_eff > 4096) return NYS_EINVAL;
    auto go = [&](auto* tu, auto* tt, auto* ta) -> int {
        using TU = std::remove_pointer_t<decltype(tu)>;
        using T = std::remove_pointer_t<decltype(tt)>;
        using TA = std::remove_pointer_t<decltype(ta)>;
        const T* sp = (const T*)s;
        T* op = (T*)out;
        T* qp = (T*)Q;
        switch (reg) {
            case NYS_REG_TV: return fused_typed<TU, T, TA, NYS_REG_TV>(ctx, pc, lb, n_inner, n1, n2, sp, op, qp);
            case NYS_REG_ISOTV: return fused_typed<TU, T, TA, NYS_REG_ISOTV>(ctx, pc, lb, n_inner, n1, n2, sp, op, qp);
            case NYS_REG_HS: return fused_typed<TU, T, TA, NYS_REG_HS>(ctx, pc, lb, n_inner, n1, n2, sp, op, qp);
            case NYS_REG_HS2: return fused_typed<TU, T, TA, NYS_REG_HS2>(ctx, pc, lb, n_inner, n1, n2, sp, op, qp);
            case NYS_REG_HSINF: return fused_typed<TU, T, TA, NYS_REG_HSINF>(ctx, pc, lb, n_inner, n1, n2, sp, op, qp);
        }
        return NYS_EINVAL;
    };
    if (dtype == NYS_F64) {
        if (pc->dtype != NYS_F64) return NYS_EINVAL;
        return go((double*)nullptr, (double*)nullptr, (double*)nullptr);
    }
    if (pc->dtype == NYS_BF16) return go((__nv_bfloat16*)nullptr, (float*)nullptr, (float*)nullptr);
    if (pc->dtype == NYS_F32) return go((float*)nullptr, (float*)nullptr, (float*)nullptr);
    return NYS_EINVAL;
}

}  // namespace nys
