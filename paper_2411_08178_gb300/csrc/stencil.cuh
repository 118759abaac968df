// Periodic difference stencils of the regularisers (Appendix A): L^T Q at one
// pixel for the first differences (anisotropic TV) and the second differences
// (Hessian), shared by the prox kernels and the unrolled-solve kernels.
#pragma once

#include "internal.cuh"

namespace nys {

template <class T>
__device__ __forceinline__ T at(const T* p, int i, int j, int n1, int n2) {
    return p[(size_t)pmod(i, n1) * n2 + pmod(j, n2)];
}

__device__ __forceinline__ int wrap_dec(int i, int n) { return i == 0 ? n - 1 : i - 1; }
__device__ __forceinline__ int wrap_inc(int i, int n) { return i + 1 == n ? 0 : i + 1; }
// row and column of flat pixel t (images hold fewer than 2^31 pixels)
__device__ __forceinline__ void pix_ij(int64_t t, int n2, int& i, int& j) {
    const unsigned u = (unsigned)t;
    i = (int)(u / (unsigned)n2);
    j = (int)(u - (unsigned)i * (unsigned)n2);
}

// first differences (anisotropic and isotropic TV) or the 2x2 Hessian
__host__ __device__ constexpr bool first_order(int reg) { return reg == NYS_REG_TV || reg == NYS_REG_ISOTV; }
// dual components per pixel
__host__ __device__ constexpr int dual_components(int reg) { return first_order(reg) ? 2 : 3; }

// L^T Q at pixel (i, j)
template <class T, int REG>
__device__ __forceinline__ typename Comp<T>::type lt_q(const T* __restrict__ Q, int i, int j, int n1, int n2) {
    using TC = typename Comp<T>::type;
    const size_t N = (size_t)n1 * n2;
    const size_t r0 = (size_t)i * n2;
    const int jp = wrap_inc(j, n2);
    const size_t rp = (size_t)wrap_inc(i, n1) * n2;
    if (first_order(REG)) {
        const T* q1 = Q;
        const T* q2 = Q + N;
        return (TC)q1[r0 + j] - (TC)q1[rp + j] + (TC)q2[r0 + j] - (TC)q2[r0 + jp];
    } else {
        const T* q11 = Q;
        const T* q12 = Q + N;
        const T* q22 = Q + 2 * N;
        const int jm = wrap_dec(j, n2);
        const size_t rm = (size_t)wrap_dec(i, n1) * n2;
        const TC a11 = (TC)q11[rm + j] - TC(2) * (TC)q11[r0 + j] + (TC)q11[rp + j];
        const TC a22 = (TC)q22[r0 + jm] - TC(2) * (TC)q22[r0 + j] + (TC)q22[r0 + jp];
        const TC a12 = TC(0.25) * ((TC)q12[rp + jp] - (TC)q12[rp + jm] - (TC)q12[rm + jp] + (TC)q12[rm + jm]);
        return a11 + TC(2) * a12 + a22;
    }
}

// One APG step of the dual at pixel t (components at t, t + N, t + 2N) given
// L x there (2 components for TV, (v11, v12, v22) for the Hessian):
// Q' = Proj(R + step L x), R <- Q' + beta (Q' - Qp), Qp <- Q'.  Proj is the
// projection onto the pixel's dual ball (Eq. mixedUnitNormBall): clip to
// [-1, 1] (anisotropic TV), scale to Euclidean norm <= 1 (isotropic TV), clip
// the eigenvalues of the symmetric 2 x 2 block (HS_1), scale it to Frobenius
// norm <= 1 (HS_2), or move its eigenvalue pair onto the l1 unit ball
// (HS_inf).  chg: set when the new Q at the pixel differs from the old R or
// Q there (the test of the exact early stop, internal.cuh).
template <class T, int REG>
__device__ __forceinline__ void dual_pixel(const typename Comp<T>::type* Lx, T* __restrict__ R, T* __restrict__ Qp,
                                           int64_t t, int64_t N, typename Comp<T>::type step,
                                           typename Comp<T>::type beta, bool* chg = nullptr) {
    using TC = typename Comp<T>::type;
    auto note = [&](TC q, TC r, TC o) {
        if (chg && !(q == r && q == o)) *chg = true;
    };
    if (REG == NYS_REG_TV) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int64_t e = t + c * N;
            const TC r = (TC)R[e];
            const TC q = fmin(TC(1), fmax(TC(-1), r + step * Lx[c]));
            const TC o = (TC)Qp[e];
            note(q, r, o);
            R[e] = (T)(q + beta * (q - o));
            Qp[e] = (T)q;
        }
    } else if (REG == NYS_REG_ISOTV) {
        TC q[2], r[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            r[c] = (TC)R[t + c * N];
            q[c] = r[c] + step * Lx[c];
        }
        const TC den = fmax(TC(1), sqrt(q[0] * q[0] + q[1] * q[1]));
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int64_t e = t + c * N;
            const TC qc = q[c] / den;
            const TC o = (TC)Qp[e];
            note(qc, r[c], o);
            R[e] = (T)(qc + beta * (qc - o));
            Qp[e] = (T)qc;
        }
    } else {
        const TC ra = (TC)R[t], rb = (TC)R[t + N], rc = (TC)R[t + 2 * N];
        const TC a = ra + step * Lx[0];
        const TC b = rb + step * Lx[1];
        const TC c = rc + step * Lx[2];
        TC pa, pb, pc;
        if (REG == NYS_REG_HS2) {
            const TC den = fmax(TC(1), sqrt(a * a + TC(2) * b * b + c * c));
            pa = a / den;
            pb = b / den;
            pc = c / den;
        } else {
            // eigenvalues m +- r of [[a, b], [b, c]], projected, recomposed on
            // the same eigenvectors
            const TC m = TC(0.5) * (a + c), h = TC(0.5) * (a - c);
            const TC r = sqrt(h * h + b * b);
            TC l1, l2;
            if (REG == NYS_REG_HSINF) {
                // onto |l1| + |l2| <= 1: soft-threshold both magnitudes by theta
                const TC e1 = m + r, e2 = m - r;
                const TC a1 = fabs(e1), a2 = fabs(e2);
                const TC big = fmax(a1, a2), small = fmin(a1, a2);
                TC th = big - small >= TC(1) ? big - TC(1) : TC(0.5) * (big + small - TC(1));
                if (a1 + a2 <= TC(1)) th = TC(0);
                l1 = copysign(fmax(a1 - th, TC(0)), e1);
                l2 = copysign(fmax(a2 - th, TC(0)), e2);
            } else {
                l1 = fmin(TC(1), fmax(TC(-1), m + r));
                l2 = fmin(TC(1), fmax(TC(-1), m - r));
            }
            const TC mp = TC(0.5) * (l1 + l2), dp = TC(0.5) * (l1 - l2);
            if (r > TC(0)) {
                pa = mp + dp * (h / r);
                pb = dp * (b / r);
                pc = mp - dp * (h / r);
            } else {
                pa = mp;
                pb = TC(0);
                pc = mp;
            }
        }
        const TC oa = (TC)Qp[t], ob = (TC)Qp[t + N], oc = (TC)Qp[t + 2 * N];
        note(pa, ra, oa);
        note(pb, rb, ob);
        note(pc, rc, oc);
        R[t] = (T)(pa + beta * (pa - oa));
        R[t + N] = (T)(pb + beta * (pb - ob));
        R[t + 2 * N] = (T)(pc + beta * (pc - oc));
        Qp[t] = (T)pa;
        Qp[t + N] = (T)pb;
        Qp[t + 2 * N] = (T)pc;
    }
}

// Inputs and outputs of one anisotropic-TV dual step fused with the L^T that
// follows it: the old (R, Q) are read from Ro/Qo and the new ones written to
// Rn/Qn (other buffers: a CTA recomputes the new values of its neighbours, so
// nothing may be overwritten in place); Rn null = the last step, which keeps
// only Q.
template <class T>
struct TvDual {
    const T* x;
    const T* Ro;
    const T* Qo;
    T* Rn;
    T* Qn;
    typename Comp<T>::type step, beta;
};

// Anisotropic TV: the dual step at pixel (i, j) and L^T of its result there.
// L x is the pair of backward differences, so the new R at (i, j) needs x at
// (i, j), (i-1, j), (i, j-1); L^T needs the new first component at (i+1, j)
// and the new second one at (i, j+1), recomputed here from x, Ro and Qo (the
// projection is a clip per component, so each needs only its own inputs).
// Writes the new (R, Q) at (i, j) and returns L^T R_new (L^T Q_new on the
// last step).  The storage type is the compute type here (float32 or
// float64 iterates), and explicit fma keeps the recomputed neighbour values
// bit-identical to the ones their own pixel writes.
// xf(q) gives x at flat index q (from memory, or from a staged copy).
// chg (not on the last step): set when the new (R, Q) at (i, j) differs
// from the old one (the test of the exact early stop, internal.cuh).
template <class T, class XF>
__device__ __forceinline__ typename Comp<T>::type tv_dual_lt_f(const TvDual<T>& d, XF xf, int i, int j, int n1,
                                                               int n2, bool* chg = nullptr) {
    using TC = typename Comp<T>::type;
    const size_t N = (size_t)n1 * n2;
    const size_t r0 = (size_t)i * n2, rm = (size_t)wrap_dec(i, n1) * n2, rp = (size_t)wrap_inc(i, n1) * n2;
    const int jm = wrap_dec(j, n2), jp = wrap_inc(j, n2);
    const size_t t = r0 + j, td = rp + j, tr = r0 + jp;
    const TC xc = xf(t);
    const TC lx1 = xc - xf(rm + j), lx1d = xf(td) - xc;
    const TC lx2 = xc - xf(r0 + jm), lx2r = xf(tr) - xc;
    // the old (R, Q) at the pixel, read once before any store (the pointers
    // may alias as far as the compiler knows)
    const TC ro1 = (TC)d.Ro[t], ro2 = (TC)d.Ro[N + t];
    const TC qo1 = d.Rn ? (TC)d.Qo[t] : TC(0), qo2 = d.Rn ? (TC)d.Qo[N + t] : TC(0);
    auto clip = [&](TC lx, TC r) { return fmin(TC(1), fmax(TC(-1), fma(d.step, lx, r))); };
    auto proj = [&](size_t e, TC lx) { return clip(lx, (TC)d.Ro[e]); };
    const TC q1 = clip(lx1, ro1), q1d = proj(td, lx1d);
    const TC q2 = clip(lx2, ro2), q2r = proj(N + tr, lx2r);
    TC mq1d = TC(0), mq2r = TC(0);
    if (d.Rn) {
        auto mom = [&](size_t e, TC q) { return fma(d.beta, q - (TC)d.Qo[e], q); };
        mq1d = mom(td, q1d);
        mq2r = mom(N + tr, q2r);
    }
    d.Qn[t] = (T)q1;
    d.Qn[N + t] = (T)q2;
    if (!d.Rn) return q1 - q1d + q2 - q2r;
    const TC r1 = fma(d.beta, q1 - qo1, q1), r2 = fma(d.beta, q2 - qo2, q2);
    d.Rn[t] = (T)r1;
    d.Rn[N + t] = (T)r2;
    if (chg && !(q1 == ro1 && q1 == qo1 && q2 == ro2 && q2 == qo2)) *chg = true;
    return r1 - mq1d + r2 - mq2r;
}
template <class T>
__device__ __forceinline__ typename Comp<T>::type tv_dual_lt(const TvDual<T>& d, int i, int j, int n1, int n2,
                                                             bool* chg = nullptr) {
    using TC = typename Comp<T>::type;
    return tv_dual_lt_f<T>(d, [&](size_t q) { return (TC)d.x[q]; }, i, j, n1, n2, chg);
}

// A skipped last dual step: the fixed point's Q out (both components)
template <class T>
__device__ __forceinline__ void tv_dual_copy_q(const TvDual<T>& d, size_t t, size_t N) {
    d.Qn[t] = d.Qo[t];
    d.Qn[N + t] = d.Qo[N + t];
}

namespace {

// Q' = Proj(R + step * L x); R <- Q' + beta (Q' - Qp); Qp <- Q' over the image
// (x read from global memory with its periodic neighbours)
// With the exact early stop (internal.cuh) this kernel keeps the step's
// flags; a skipped step does nothing (R and Q are updated in place, so they
// already hold the fixed point).
template <class T, int REG>
__global__ void dual_update_kernel(const T* __restrict__ x, T* __restrict__ R, T* __restrict__ Qp,
                                   typename Comp<T>::type step, typename Comp<T>::type beta, int n1, int n2,
                                   DualStop stop) {
    pdl_enter();
    using TC = typename Comp<T>::type;
    const int64_t N = (int64_t)n1 * n2;
    const bool skip = dual_skip(stop);
    dual_stop_enter(stop, skip);
    if (skip) return;
    bool chg = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        int i, j;
        pix_ij(t, n2, i, j);
        const size_t r0 = (size_t)i * n2, rm = (size_t)wrap_dec(i, n1) * n2;
        const int jm = wrap_dec(j, n2);
        const TC xc = (TC)x[t];
        TC Lx[3];
        if (first_order(REG)) {
            Lx[0] = xc - (TC)x[rm + j];
            Lx[1] = xc - (TC)x[r0 + jm];
            Lx[2] = TC(0);
        } else {
            const size_t rp = (size_t)wrap_inc(i, n1) * n2;
            const int jp = wrap_inc(j, n2);
            Lx[0] = (TC)x[rm + j] - TC(2) * xc + (TC)x[rp + j];
            Lx[2] = (TC)x[r0 + jm] - TC(2) * xc + (TC)x[r0 + jp];
            Lx[1] = TC(0.25) * ((TC)x[rp + jp] - (TC)x[rp + jm] - (TC)x[rm + jp] + (TC)x[rm + jm]);
        }
        dual_pixel<T, REG>(Lx, R, Qp, t, N, step, beta, &chg);
    }
    dual_stop_report(stop, chg);
}

}  // namespace

}  // namespace nys
