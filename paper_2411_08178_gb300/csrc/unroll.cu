// Differentiated unrolled solve: K iterations of Algorithm 3 with the
// anisotropic TV regulariser (dual APG prox of Sec. III-B, n_inner steps,
// warm-started dual), and a hand-written reverse pass giving the gradient of
// <xbar, x_K> with respect to lambda and to the blur kernel h.
//
// Forward, per outer iteration k (lb = alpha lambda, step = 1 / (8 lb)):
//     r_k = A u_k - y,  s = u_k - alpha P^{-1} A^T r_k
//     j = 0 .. J-1:  x_j = s - lb P^{-1} L^T R_j
//                    z_j = R_j + step L x_j,  Q_{j+1} = clip(z_j, -1, 1)
//                    R_{j+1} = Q_{j+1} + beta_j (Q_{j+1} - Q_j)
//     x_{k+1} = s - lb P^{-1} L^T Q_J,  u_{k+1} = x_{k+1} + gamma_k (x_{k+1} - x_k)
// P and alpha are constants of the map.  The forward keeps (x, u, Q) every
// `ckpt_every` iterations; the backward re-runs one segment at a time from
// its checkpoint, recording u_k, r_k, Q_0 and every z_j (Q_{j+1} = clip(z_j),
// R_j follows from the Q's), and then walks the segment backwards:
//     xbar_{k+1} += (1 + gamma_k) ubar_{k+1};  xbar_k = -gamma_k ubar_{k+1}
//     sbar = xbar_{k+1};  Qbar_J = Qbar_warm - lb L P^{-1} xbar_{k+1}
//     j = J-1 .. 0:  zbar = 1[|z_j| < 1] (Qbar_{j+1} + (1 + beta_j) Rbar_{j+1})
//                    Qbar_j = -beta_j Rbar_{j+1}
//                    sbar += step L^T zbar,  w = P^{-1} L^T zbar
//                    Rbar_j = zbar - (1/8) L w
//     Qbar_warm = Qbar_0 + Rbar_0
//     t = P^{-1} sbar;  ubar_k = sbar - alpha A^T A t
//     dh += -alpha (dK(r_k, t) + dK(A t, u_k)),  dK(w, x)[a,b] = sum w[i,j] x[i+a-c, j+b-c]
// and d lb collects -<L P^{-1} xbar_{k+1}, Q_J>, and per dual step
// -(1/lb) <zbar, z_j - R_j> - step <L w, R_j>; d lambda = alpha d lb.
// Every reduction goes to a per-CTA float64 accumulator (fixed grid, fixed
// pixel-to-CTA map) that one final pass sums, so the result is deterministic.
#include "internal.cuh"
#include "stencil.cuh"

#include <algorithm>
#include <cmath>

struct nys_unroll {
    nys_ctx* ctx = nullptr;
    nys_op* op = nullptr;
    const nys_precond* pc = nullptr;
    int dtype = 0;
    double lambda = 0, alpha = 0;
    int K = 0, J = 0, C = 1, nseg = 0;
    int64_t N = 0, M = 0;
    int grid = 0, kgrid = 0, ntaps = 0;
    std::vector<double> gam, bet;
    bool have_fwd = false;
    // device memory (element type = dtype unless noted)
    void* y = nullptr;      // M, data of the last forward
    void* st = nullptr;     // x, u (N each), Q (2N), xn (N)
    void* ckpt = nullptr;   // nseg x (x, u, Q)
    void* rec = nullptr;    // C x (u N, r M, slots (J+1) 2N)
    void* tmp = nullptr;    // s, g, xt, R, Qp, xbar, ubar, sbar, t1, nb (N each) + R, Qp, Qbar, Rbar, Qbarw (2N) + a1 (M)
    double* acc = nullptr;  // grid (d lb partials) + kgrid * ntaps (dh partials) + 1 + ntaps (results)
};

namespace nys {
namespace {

template <class T>
struct UB {
    using TC = typename Comp<T>::type;
    T *x, *u, *Q, *xn;
    T *s, *g, *xt, *xbar, *ubar, *sbar, *t1, *nb;
    T *R, *Qp, *Qbar, *Rbar, *Qbw;
    T* a1;
    T* y;
    size_t rec_stride;
    T* rec;
    T* ckpt;
    T* rec_u(int i) const { return rec + (size_t)i * rec_stride; }
    T* rec_r(int i, int64_t N) const { return rec_u(i) + N; }
    T* rec_slot(int i, int j, int64_t N, int64_t M) const { return rec_u(i) + N + M + (size_t)j * 2 * N; }
};

template <class T>
UB<T> bufs(const nys_unroll* U) {
    UB<T> b;
    const int64_t N = U->N, M = U->M;
    T* p = (T*)U->st;
    b.x = p;
    b.u = p + N;
    b.Q = p + 2 * N;
    b.xn = p + 4 * N;
    T* t = (T*)U->tmp;
    b.s = t; b.g = t + N; b.xt = t + 2 * N; b.xbar = t + 3 * N; b.ubar = t + 4 * N;
    b.sbar = t + 5 * N; b.t1 = t + 6 * N; b.nb = t + 7 * N;
    T* t2 = t + 8 * N;
    b.R = t2; b.Qp = t2 + 2 * N; b.Qbar = t2 + 4 * N; b.Rbar = t2 + 6 * N; b.Qbw = t2 + 8 * N;
    b.a1 = t2 + 10 * N;
    b.y = (T*)U->y;
    b.rec_stride = (size_t)N + M + (size_t)(U->J + 1) * 2 * N;
    b.rec = (T*)U->rec;
    b.ckpt = (T*)U->ckpt;
    return b;
}

#define GRID_LOOP(t, n) for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (n); t += (int64_t)gridDim.x * blockDim.x)

template <class T>
__device__ __forceinline__ typename Comp<T>::type clip1(T v) {
    using TC = typename Comp<T>::type;
    return fmin(TC(1), fmax(TC(-1), (TC)v));
}

// r = r - y
template <class T>
__global__ void sub_kernel(T* __restrict__ r, const T* __restrict__ y, int64_t n) {
    GRID_LOOP(t, n) r[t] = r[t] - y[t];
}

// out = a + c * b
template <class T>
__global__ void axpy_kernel(const T* __restrict__ a, const T* __restrict__ b, double c, int64_t n, T* __restrict__ out) {
    using TC = typename Comp<T>::type;
    GRID_LOOP(t, n) out[t] = (T)((TC)a[t] + (TC)c * (TC)b[t]);
}

// out = L^T Q (TV); if acc_into: acc_into += c * out
template <class T>
__global__ void lt_tv_kernel(const T* __restrict__ Q, int n1, int n2, T* __restrict__ out, T* __restrict__ acc_into,
                             double c) {
    using TC = typename Comp<T>::type;
    const int64_t N = (int64_t)n1 * n2;
    GRID_LOOP(t, N) {
        const int i = (int)(t / n2), j = (int)(t - (int64_t)i * n2);
        const TC g = lt_q<T, NYS_REG_TV>(Q, i, j, n1, n2);
        out[t] = (T)g;
        if (acc_into) acc_into[t] = (T)((TC)acc_into[t] + (TC)c * g);
    }
}

// forward dual step: z = R + step L x; Q' = clip(z); R <- Q' + beta (Q' - Qp);
// Qp <- Q'; z stored if zout
template <class T>
__global__ void dual_step_kernel(const T* __restrict__ x, T* __restrict__ R, T* __restrict__ Qp,
                                 T* __restrict__ zout, double step, double beta, int n1, int n2) {
    using TC = typename Comp<T>::type;
    const int64_t N = (int64_t)n1 * n2;
    GRID_LOOP(t, N) {
        const int i = (int)(t / n2), j = (int)(t - (int64_t)i * n2);
        const TC xc = (TC)x[t];
        const TC v[2] = {xc - (TC)at(x, i - 1, j, n1, n2), xc - (TC)at(x, i, j - 1, n1, n2)};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int64_t e = t + c * N;
            const T z = (T)((TC)R[e] + (TC)step * v[c]);
            const TC q = clip1(z);
            const TC o = (TC)Qp[e];
            R[e] = (T)(q + (TC)beta * (q - o));
            Qp[e] = (T)q;
            if (zout) zout[e] = z;
        }
    }
}

// u = xn + gamma (xn - x); x = xn
template <class T>
__global__ void momentum_kernel(const T* __restrict__ xn, T* __restrict__ x, T* __restrict__ u, double gamma,
                                int64_t N) {
    using TC = typename Comp<T>::type;
    GRID_LOOP(t, N) {
        const TC a = (TC)xn[t], b = (TC)x[t];
        u[t] = (T)(a + (TC)gamma * (a - b));
        x[t] = (T)a;
    }
}

// ----------------------------------------------------------- backward ----
template <class T>
__device__ __forceinline__ void acc_add(double v, double* acc, double* sh) {
    const double s = block_sum(v, sh);
    if (threadIdx.x == 0) acc[blockIdx.x] += s;
}

// sbar = xbar + (1 + g) ubar;  xbar <- -g ubar
template <class T>
__global__ void mom_bwd_kernel(T* __restrict__ xbar, const T* __restrict__ ubar, T* __restrict__ sbar, double g,
                               int64_t N) {
    using TC = typename Comp<T>::type;
    GRID_LOOP(t, N) {
        const TC ub = (TC)ubar[t];
        sbar[t] = (T)((TC)xbar[t] + (TC)(1.0 + g) * ub);
        xbar[t] = (T)(-(TC)g * ub);
    }
}

// Qbar = Qbw - lb L w;  acc += -<L w, clip(QJ)>;  Rbar = 0
template <class T>
__global__ void __launch_bounds__(256) out_bwd_kernel(const T* __restrict__ w, const T* __restrict__ Qbw,
                                                      const T* __restrict__ QJ, double lb, int n1, int n2,
                                                      T* __restrict__ Qbar, T* __restrict__ Rbar,
                                                      double* __restrict__ acc) {
    using TC = typename Comp<T>::type;
    __shared__ double sh[32];
    const int64_t N = (int64_t)n1 * n2;
    double part = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / n2), j = (int)(t - (int64_t)i * n2);
        const TC wc = (TC)w[t];
        const TC Lw[2] = {wc - (TC)at(w, i - 1, j, n1, n2), wc - (TC)at(w, i, j - 1, n1, n2)};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int64_t e = t + c * N;
            Qbar[e] = (T)((TC)Qbw[e] - (TC)lb * Lw[c]);
            Rbar[e] = T(0);
            part -= (double)Lw[c] * (double)clip1(QJ[e]);
        }
    }
    acc_add<T>(part, acc, sh);
}

// zbar = 1[|z| < 1] (Qbar + (1 + beta) Rbar);  Qbar <- -beta Rbar;  Rbar <- zbar
template <class T>
__global__ void zbar_kernel(T* __restrict__ Qbar, T* __restrict__ Rbar, const T* __restrict__ z, double beta,
                            int64_t n) {
    using TC = typename Comp<T>::type;
    GRID_LOOP(t, n) {
        const TC rb = (TC)Rbar[t];
        const TC qb = (TC)Qbar[t] + (TC)(1.0 + beta) * rb;
        const TC zz = (TC)z[t];
        Rbar[t] = (T)((zz < TC(1) && zz > TC(-1)) ? qb : TC(0));
        Qbar[t] = (T)(-(TC)beta * rb);
    }
}

// Rbar <- zbar - (1/8) L w (w = P^{-1} L^T zbar, before the step factor);
// acc += -(1/lb) <zbar, z - R_j> - step <L w, R_j>, with R_j from the slots
// (R_0 = Q_0, R_j = (1 + b) clip(slot_j) - b clip(slot_{j-1}), b = beta_{j-1})
template <class T>
__global__ void __launch_bounds__(256) rbar_kernel(const T* __restrict__ w, const T* __restrict__ z,
                                                   const T* __restrict__ Sj, const T* __restrict__ Sjm,
                                                   double bprev, double lb, double step, int n1, int n2,
                                                   T* __restrict__ Rbar, double* __restrict__ acc) {
    using TC = typename Comp<T>::type;
    __shared__ double sh[32];
    const int64_t N = (int64_t)n1 * n2;
    double part = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / n2), j = (int)(t - (int64_t)i * n2);
        const TC wc = (TC)w[t];
        const TC Lw[2] = {wc - (TC)at(w, i - 1, j, n1, n2), wc - (TC)at(w, i, j - 1, n1, n2)};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int64_t e = t + c * N;
            const TC qj = clip1(Sj[e]);
            const TC Rj = Sjm ? (TC)(1.0 + bprev) * qj - (TC)bprev * clip1(Sjm[e]) : qj;
            const TC zb = (TC)Rbar[e];
            part -= (double)zb * ((double)z[e] - (double)Rj) / lb + step * (double)Lw[c] * (double)Rj;
            Rbar[e] = (T)(zb - TC(0.125) * Lw[c]);
        }
    }
    acc_add<T>(part, acc, sh);
}

// out += scale * dK(w, x): the derivative of <w, h (*) x> with respect to each
// tap, for one 32 x 32 pixel tile per CTA (x staged with its halo); the
// per-CTA partials are kept in float64 and summed by the final pass
constexpr int KT = 32;
template <class T>
__global__ void __launch_bounds__(256) kgrad_kernel(const T* __restrict__ w, const T* __restrict__ x, int n1, int n2,
                                                    int kh, int kw, double scale, double* __restrict__ part) {
    using TC = typename Comp<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ch = (kh - 1) / 2, cw = (kw - 1) / 2;
    const int tiles2 = (n2 + KT - 1) / KT;
    const int i0 = (blockIdx.x / tiles2) * KT, j0 = (blockIdx.x % tiles2) * KT;
    const int hw = KT + kw - 1, hh = KT + kh - 1;
    TC* ws = reinterpret_cast<TC*>(smem_raw);   // KT x KT
    TC* xs = ws + KT * KT;                      // hh x hw, xs[p][q] = x[i0 + p - ch][j0 + q - cw]
    for (int t = threadIdx.x; t < KT * KT; t += blockDim.x) {
        const int i = i0 + t / KT, j = j0 + t % KT;
        ws[t] = (i < n1 && j < n2) ? (TC)w[(size_t)i * n2 + j] : TC(0);
    }
    for (int t = threadIdx.x; t < hh * hw; t += blockDim.x) {
        const int p = t / hw, q = t % hw;
        xs[t] = (TC)at(x, i0 + p - ch, j0 + q - cw, n1, n2);
    }
    __syncthreads();
    const int ntaps = kh * kw;
    for (int tap = threadIdx.x; tap < ntaps; tap += blockDim.x) {
        const int a = tap / kw, b = tap % kw;
        TC s = TC(0);
        for (int pi = 0; pi < KT; ++pi) {
            const TC* wr = ws + pi * KT;
            const TC* xr = xs + (pi + a) * hw + b;
#pragma unroll 8
            for (int pj = 0; pj < KT; ++pj) s = fma(wr[pj], xr[pj], s);
        }
        part[(size_t)blockIdx.x * ntaps + tap] += scale * (double)s;
    }
}

// dlam = alpha * sum(acc);  dh[tap] = sum over CTAs of the tap partials
__global__ void final_kernel(const double* __restrict__ acc, int grid, const double* __restrict__ kpart, int kgrid,
                             int ntaps, double alpha, double* __restrict__ out) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int t = threadIdx.x; t < grid; t += blockDim.x) v += acc[t];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) out[0] = alpha * v;
    for (int tap = threadIdx.x; tap < ntaps; tap += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < kgrid; ++b) s += kpart[(size_t)b * ntaps + tap];
        out[1 + tap] = s;
    }
}

// ---------------------------------------------------------------- host ---
template <class T>
int pinv(nys_unroll* U, const T* z, T* out) {
    if (!U->pc) {
        if (z != out) NYS_CK(U->ctx, cudaMemcpyAsync(out, z, sizeof(T) * U->N, cudaMemcpyDeviceToDevice, U->ctx->stream));
        return NYS_OK;
    }
    return precond_run(U->ctx, U->pc, 1, U->dtype, z, out, 1);
}

// one forward outer iteration k; rec_i >= 0 records into record slot rec_i
template <class T>
int fwd_iter(nys_unroll* U, const UB<T>& b, int k, int rec_i) {
    nys_ctx* ctx = U->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t N = U->N, M = U->M;
    const int n1 = U->op->n1, n2 = U->op->n2;
    const double lb = U->alpha * U->lambda, step = 1.0 / (8.0 * lb);
    const int g = U->grid;
    int st;
    T* r = rec_i >= 0 ? b.rec_r(rec_i, N) : b.a1;
    if (rec_i >= 0) NYS_CK(ctx, cudaMemcpyAsync(b.rec_u(rec_i), b.u, sizeof(T) * N, cudaMemcpyDeviceToDevice, s));
    if ((st = op_run(U->op, 0, b.u, r, 1, U->dtype, U->dtype))) return st;
    sub_kernel<T><<<g, 256, 0, s>>>(r, b.y, M);
    NYS_LAUNCH_CK(ctx);
    if ((st = op_run(U->op, 1, r, b.g, 1, U->dtype, U->dtype))) return st;
    if ((st = pinv<T>(U, b.g, b.g))) return st;
    axpy_kernel<T><<<g, 256, 0, s>>>(b.u, b.g, -U->alpha, N, b.s);
    NYS_LAUNCH_CK(ctx);
    if (rec_i >= 0)
        NYS_CK(ctx, cudaMemcpyAsync(b.rec_slot(rec_i, 0, N, M), b.Q, sizeof(T) * 2 * N, cudaMemcpyDeviceToDevice, s));
    NYS_CK(ctx, cudaMemcpyAsync(b.R, b.Q, sizeof(T) * 2 * N, cudaMemcpyDeviceToDevice, s));
    NYS_CK(ctx, cudaMemcpyAsync(b.Qp, b.Q, sizeof(T) * 2 * N, cudaMemcpyDeviceToDevice, s));
    for (int j = 0; j < U->J; ++j) {
        lt_tv_kernel<T><<<g, 256, 0, s>>>(b.R, n1, n2, b.g, nullptr, 0.0);
        NYS_LAUNCH_CK(ctx);
        if ((st = pinv<T>(U, b.g, b.g))) return st;
        axpy_kernel<T><<<g, 256, 0, s>>>(b.s, b.g, -lb, N, b.xt);
        NYS_LAUNCH_CK(ctx);
        T* z = rec_i >= 0 ? b.rec_slot(rec_i, j + 1, N, M) : nullptr;
        dual_step_kernel<T><<<g, 256, 0, s>>>(b.xt, b.R, b.Qp, z, step, U->bet[j], n1, n2);
        NYS_LAUNCH_CK(ctx);
    }
    NYS_CK(ctx, cudaMemcpyAsync(b.Q, b.Qp, sizeof(T) * 2 * N, cudaMemcpyDeviceToDevice, s));
    lt_tv_kernel<T><<<g, 256, 0, s>>>(b.Q, n1, n2, b.g, nullptr, 0.0);
    NYS_LAUNCH_CK(ctx);
    if ((st = pinv<T>(U, b.g, b.g))) return st;
    axpy_kernel<T><<<g, 256, 0, s>>>(b.s, b.g, -lb, N, b.xn);
    NYS_LAUNCH_CK(ctx);
    momentum_kernel<T><<<g, 256, 0, s>>>(b.xn, b.x, b.u, U->gam[k], N);
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

template <class T>
T* ckpt_ptr(const nys_unroll* U, const UB<T>& b, int seg) {
    return b.ckpt + (size_t)seg * 4 * U->N;   // x, u, Q
}

template <class T>
int forward_typed(nys_unroll* U, const void* y, void* x_out) {
    nys_ctx* ctx = U->ctx;
    cudaStream_t s = ctx->stream;
    UB<T> b = bufs<T>(U);
    const int64_t N = U->N;
    NYS_CK(ctx, cudaMemcpyAsync(b.y, y, sizeof(T) * U->M, cudaMemcpyDeviceToDevice, s));
    NYS_CK(ctx, cudaMemsetAsync(b.x, 0, sizeof(T) * 4 * N, s));   // x, u, Q
    int st;
    for (int k = 0; k < U->K; ++k) {
        if (k % U->C == 0)
            NYS_CK(ctx, cudaMemcpyAsync(ckpt_ptr(U, b, k / U->C), b.x, sizeof(T) * 4 * N, cudaMemcpyDeviceToDevice, s));
        if ((st = fwd_iter<T>(U, b, k, -1))) return st;
    }
    if (x_out) NYS_CK(ctx, cudaMemcpyAsync(x_out, b.x, sizeof(T) * N, cudaMemcpyDeviceToDevice, s));
    U->have_fwd = true;
    return NYS_OK;
}

template <class T>
int backward_typed(nys_unroll* U, const void* xbar_in, double* grads) {
    nys_ctx* ctx = U->ctx;
    cudaStream_t s = ctx->stream;
    UB<T> b = bufs<T>(U);
    const int64_t N = U->N, M = U->M;
    const int n1 = U->op->n1, n2 = U->op->n2;
    const double lb = U->alpha * U->lambda, step = 1.0 / (8.0 * lb);
    const int g = U->grid, J = U->J;
    const bool want_h = U->op->kind == NYS_OP_BLUR;
    double* acc = U->acc;
    double* kpart = acc + g;
    int st;
    NYS_CK(ctx, cudaMemsetAsync(acc, 0, sizeof(double) * ((size_t)g + (size_t)U->kgrid * U->ntaps), s));
    NYS_CK(ctx, cudaMemcpyAsync(b.xbar, xbar_in, sizeof(T) * N, cudaMemcpyDeviceToDevice, s));
    NYS_CK(ctx, cudaMemsetAsync(b.ubar, 0, sizeof(T) * N, s));
    NYS_CK(ctx, cudaMemsetAsync(b.Qbw, 0, sizeof(T) * 2 * N, s));
    const size_t ksmem = sizeof(typename Comp<T>::type) *
                         ((size_t)KT * KT + (size_t)(KT + U->op->kh - 1) * (KT + U->op->kw - 1));
    for (int seg = U->nseg - 1; seg >= 0; --seg) {
        const int k0 = seg * U->C, k1 = std::min(U->K, k0 + U->C);
        NYS_CK(ctx, cudaMemcpyAsync(b.x, ckpt_ptr(U, b, seg), sizeof(T) * 4 * N, cudaMemcpyDeviceToDevice, s));
        for (int k = k0; k < k1; ++k)
            if ((st = fwd_iter<T>(U, b, k, k - k0))) return st;
        for (int k = k1 - 1; k >= k0; --k) {
            const int ri = k - k0;
            mom_bwd_kernel<T><<<g, 256, 0, s>>>(b.xbar, b.ubar, b.sbar, U->gam[k], N);
            NYS_LAUNCH_CK(ctx);
            if ((st = pinv<T>(U, b.sbar, b.g))) return st;
            out_bwd_kernel<T><<<g, 256, 0, s>>>(b.g, b.Qbw, b.rec_slot(ri, J, N, M), lb, n1, n2, b.Qbar, b.Rbar, acc);
            NYS_LAUNCH_CK(ctx);
            for (int j = J - 1; j >= 0; --j) {
                zbar_kernel<T><<<g, 256, 0, s>>>(b.Qbar, b.Rbar, b.rec_slot(ri, j + 1, N, M), U->bet[j], 2 * N);
                NYS_LAUNCH_CK(ctx);
                lt_tv_kernel<T><<<g, 256, 0, s>>>(b.Rbar, n1, n2, b.g, b.sbar, step);
                NYS_LAUNCH_CK(ctx);
                if ((st = pinv<T>(U, b.g, b.g))) return st;
                const T* Sjm = j >= 1 ? b.rec_slot(ri, j - 1, N, M) : nullptr;
                const double bprev = j >= 1 ? U->bet[j - 1] : 0.0;
                rbar_kernel<T><<<g, 256, 0, s>>>(b.g, b.rec_slot(ri, j + 1, N, M), b.rec_slot(ri, j, N, M), Sjm,
                                                 bprev, lb, step, n1, n2, b.Rbar, acc);
                NYS_LAUNCH_CK(ctx);
            }
            axpy_kernel<T><<<g, 256, 0, s>>>(b.Qbar, b.Rbar, 1.0, 2 * N, b.Qbw);
            NYS_LAUNCH_CK(ctx);
            // ubar_k = sbar - alpha A^T A P^{-1} sbar
            if ((st = pinv<T>(U, b.sbar, b.t1))) return st;
            if ((st = op_run(U->op, 0, b.t1, b.a1, 1, U->dtype, U->dtype))) return st;
            if ((st = op_run(U->op, 1, b.a1, b.nb, 1, U->dtype, U->dtype))) return st;
            axpy_kernel<T><<<g, 256, 0, s>>>(b.sbar, b.nb, -U->alpha, N, b.ubar);
            NYS_LAUNCH_CK(ctx);
            if (want_h) {
                kgrad_kernel<T><<<U->kgrid, 256, ksmem, s>>>(b.rec_r(ri, N), b.t1, n1, n2, U->op->kh, U->op->kw,
                                                             -U->alpha, kpart);
                NYS_LAUNCH_CK(ctx);
                kgrad_kernel<T><<<U->kgrid, 256, ksmem, s>>>(b.a1, b.rec_u(ri), n1, n2, U->op->kh, U->op->kw,
                                                             -U->alpha, kpart);
                NYS_LAUNCH_CK(ctx);
            }
        }
    }
    final_kernel<<<1, 256, 0, s>>>(acc, g, kpart, want_h ? U->kgrid : 0, want_h ? U->ntaps : 0, U->alpha,
                                   acc + g + (size_t)U->kgrid * U->ntaps);
    NYS_LAUNCH_CK(ctx);
    NYS_CK(ctx, cudaMemcpyAsync(grads, acc + g + (size_t)U->kgrid * U->ntaps, sizeof(double) * (1 + (want_h ? U->ntaps : 0)),
                                cudaMemcpyDeviceToDevice, s));
    return NYS_OK;
}

std::vector<double> tseq(int count) {
    std::vector<double> out;
    double tp = 1.0;
    for (int k = 0; k < count; ++k) {
        const double t = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * tp * tp));
        out.push_back((tp - 1.0) / t);
        tp = t;
    }
    return out;
}

}  // namespace
}  // namespace nys

namespace nys {
// the contexts an unrolled-solve handle launches on (its own and its op's)
void unroll_contexts(const nys_unroll* U, nys_ctx** ctx, nys_ctx** op_ctx) {
    *ctx = U->ctx;
    *op_ctx = U->op->ctx;
}
}  // namespace nys

using namespace nys;

extern "C" {

int nys_unroll_create(nys_ctx* ctx, nys_op* op, const nys_precond* pc, const nys_unroll_desc* d, nys_unroll** out) {
    if (!ctx || !op || !d || !out) return fail(ctx, NYS_EINVAL, "null argument");
    *out = nullptr;
    if (op->dtype != NYS_F32 && op->dtype != NYS_F64) return fail(ctx, NYS_EINVAL, "unrolled solve needs f32 or f64");
    if (!(d->lambda > 0.0) || !(d->alpha > 0.0) || d->K < 1 || d->n_inner < 0 || d->ckpt_every < 0)
        return fail(ctx, NYS_EINVAL, "unrolled solve needs lambda > 0, alpha > 0, K >= 1, n_inner >= 0");
    if (pc && (pc->N != op->N || !pc->priv)) return fail(ctx, NYS_EINVAL, "preconditioner size mismatch or not set up");
    nys_unroll* U = new nys_unroll();
    U->ctx = ctx;
    ctx_retain(ctx);
    U->op = op;
    U->pc = pc;
    U->dtype = op->dtype;
    U->lambda = d->lambda;
    U->alpha = d->alpha;
    U->K = d->K;
    U->J = d->n_inner;
    U->C = d->ckpt_every > 0 ? std::min(d->ckpt_every, d->K) : d->K;
    U->nseg = (U->K + U->C - 1) / U->C;
    U->N = op->N;
    U->M = op->M;
    U->grid = (int)std::min<int64_t>((std::max(U->N, U->M) + 255) / 256, (int64_t)ctx->sm_count * 8);
    U->kgrid = ((op->n1 + KT - 1) / KT) * ((op->n2 + KT - 1) / KT);
    U->ntaps = op->kind == NYS_OP_BLUR ? op->kh * op->kw : 0;
    U->gam = tseq(U->K);
    U->bet = tseq(U->J);
    const size_t es = dtype_size(U->dtype);
    const size_t N = U->N, M = U->M;
    const size_t rec_stride = N + M + (size_t)(U->J + 1) * 2 * N;
    size_t kbytes = 0;
    if (U->ntaps) {
        const size_t ksm = (op->dtype == NYS_F64 ? 8 : 4) *
                           ((size_t)KT * KT + (size_t)(KT + op->kh - 1) * (KT + op->kw - 1));
        if (ksm > 227 * 1024) {
            delete U;
            return fail(ctx, NYS_EINVAL, "blur kernel too large for the kernel-gradient tile");
        }
        kbytes = ksm;
    }
    auto alloc = [&](void** p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 16)); };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = alloc(&U->y, es * M);
    if (e == cudaSuccess) e = alloc(&U->st, es * 5 * N);
    if (e == cudaSuccess) e = alloc(&U->ckpt, es * 4 * N * U->nseg);
    if (e == cudaSuccess) e = alloc(&U->rec, es * rec_stride * U->C);
    if (e == cudaSuccess) e = alloc(&U->tmp, es * (18 * N + M));
    if (e == cudaSuccess)
        e = alloc((void**)&U->acc, sizeof(double) * ((size_t)U->grid + (size_t)U->kgrid * U->ntaps + 1 + U->ntaps));
    if (e == cudaSuccess && kbytes > 48 * 1024) {
        e = op->dtype == NYS_F64 ? cudaFuncSetAttribute(kgrad_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kbytes)
                                 : cudaFuncSetAttribute(kgrad_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kbytes);
    }
    if (e != cudaSuccess) {
        nys_unroll_destroy(U);
        return cuda_fail(ctx, e, "unrolled-solve buffers");
    }
    *out = U;
    return NYS_OK;
}

int nys_unroll_destroy(nys_unroll* U) {
    if (!U) return NYS_OK;
    if (U->ctx) cudaStreamSynchronize(U->ctx->stream);
    void* bufs_[] = {U->y, U->st, U->ckpt, U->rec, U->tmp, U->acc};
    for (void* p : bufs_)
        if (p) cudaFree(p);
    nys_ctx* ctx = U->ctx;
    delete U;
    ctx_release(ctx);
    return NYS_OK;
}

int nys_unroll_forward(nys_unroll* U, const void* y, void* x_out) {
    if (!U || !y) return fail(U ? U->ctx : nullptr, NYS_EINVAL, "null argument");
    return U->dtype == NYS_F64 ? forward_typed<double>(U, y, x_out) : forward_typed<float>(U, y, x_out);
}

int nys_unroll_backward(nys_unroll* U, const void* xbar, double* grads) {
    if (!U || !xbar || !grads) return fail(U ? U->ctx : nullptr, NYS_EINVAL, "null argument");
    if (!U->have_fwd) return fail(U->ctx, NYS_EINVAL, "nys_unroll_backward before nys_unroll_forward");
    return U->dtype == NYS_F64 ? backward_typed<double>(U, xbar, grads) : backward_typed<float>(U, xbar, grads);
}

int nys_unroll_set_lambda(nys_unroll* U, double lambda) {
    if (!U || !(lambda > 0.0)) return fail(U ? U->ctx : nullptr, NYS_EINVAL, "lambda must be > 0");
    U->lambda = lambda;
    U->have_fwd = false;
    return NYS_OK;
}

}  // extern "C"
