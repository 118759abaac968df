// Weighted proximal mappings in the P metric (Sec. III-B).
//
// prox_tv / prox_hs: the dual scheme for lambda_bar ||L x||_{1,phi} with
// C = R^N.  The dual objective ||s - lb P^{-1} L^T Q||_P^2 over the unit ball of
// the dual norm has gradient -2 lb L x(Q), x(Q) = s - lb P^{-1} L^T Q, and
// Lipschitz constant 2 lb^2 ||L||^2 (sigma_min(P) = 1), so each APG (FISTA)
// step is
//     x   = s - lb P^{-1} L^T R
//     Q'  = Proj(R + L x / (lb ||L||^2))
//     R   = Q' + beta_k (Q' - Q)           beta_k from the fixed t_k sequence
// L = first differences (anisotropic TV, ||L||^2 = 8, Proj = clip to [-1,1])
// or second differences (Hessian Schatten-1, ||L||^2 = 32 in the inner
// product q11 v11 + 2 q12 v12 + q22 v22, Proj = clip the eigenvalues of each
// symmetric 2 x 2 block to [-1, 1]).  Kernels: one stencil pass for L^T R
// (fused with x = s - lb L^T R when P = I), P^{-1} through precond_run, and
// one pass that forms L x, projects and extrapolates.  beta_k depends only on
// k, so it is a kernel argument and no host synchronisation is needed.
//
// prox_wavelet: Theorem 1 with D = I, W = I + Ubar Ubar^T: out =
// T_tau(s - Ubar gamma*), gamma* solving F(gamma) = Ubar^T (s - T_tau(s - Ubar
// gamma)) + gamma = 0 by semi-smooth Newton with step halving.  The Newton
// state machine runs on the device: an evaluation pass over the pixels
// computes F (float64) and the generalised Jacobian J = I + Ubar_S^T Ubar_S on
// the support S = {|z| > tau} (float32 partial sums: J only steers the Newton
// direction, F decides the solution), and a one-CTA pass accepts or halves
// the step and solves J d = -F by Cholesky.
#include "internal.cuh"
#include "chol.cuh"
#include "stencil.cuh"

#include <cmath>

namespace nys {

namespace {

// out = base - lb * L^T Q   (base may be null -> out = L^T Q, lb ignored);
// nothing inside a dual step that the exact early stop skips
template <class T, int REG>
__global__ void lt_kernel(const T* __restrict__ Q, const T* __restrict__ base, typename Comp<T>::type lb, int n1,
                          int n2, T* __restrict__ out, DualStop stop) {
    pdl_enter();
    if (dual_skip(stop)) return;
    using TC = typename Comp<T>::type;
    const int64_t N = (int64_t)n1 * n2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        int i, j;
        pix_ij(t, n2, i, j);
        const TC g = lt_q<T, REG>(Q, i, j, n1, n2);
        out[t] = base ? (T)((TC)base[t] - lb * g) : (T)g;
    }
}

// x = s - lb * pg   (pg = P^{-1} L^T R)
template <class T>
__global__ void axpy_kernel(const T* __restrict__ s, const T* __restrict__ pg, typename Comp<T>::type lb, int64_t N,
                            T* __restrict__ x) {
    pdl_enter();
    using TC = typename Comp<T>::type;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x)
        x[t] = (T)((TC)s[t] - lb * (TC)pg[t]);
}

// Plain (P = I) anisotropic-TV dual step fused with the x after it:
// out = s - lb L^T R_new (L^T Q_new on the last step); out is not d.x.
// With the exact early stop (internal.cuh) a skipped step does nothing, a
// skipped last step writes Q and out = x (at the fixed point R = Q, so the
// two L^T agree bit for bit).
template <class T>
__global__ void tv_dual_x_kernel(TvDual<T> d, const T* __restrict__ s, typename Comp<T>::type lb, int n1, int n2,
                                 T* __restrict__ out, DualStop stop) {
    pdl_enter();
    using TC = typename Comp<T>::type;
    const int64_t N = (int64_t)n1 * n2;
    const bool skip = dual_skip(stop);
    dual_stop_enter(stop, skip);
    if (skip) {
        if (!d.Rn)
            for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
                 t += (int64_t)gridDim.x * blockDim.x) {
                tv_dual_copy_q<T>(d, (size_t)t, (size_t)N);
                out[t] = d.x[t];
            }
        return;
    }
    bool chg = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        int i, j;
        pix_ij(t, n2, i, j);
        const TC g = tv_dual_lt<T>(d, i, j, n1, n2, &chg);
        out[t] = (T)((TC)s[t] - lb * g);
    }
    dual_stop_report(stop, chg);
}

template <class T, int REG>
int prox_dual_typed(nys_ctx* ctx, const nys_precond* pc, double lb, int n_inner, int n1, int n2, const T* s, T* out,
                    T* Q) {
    using TC = typename Comp<T>::type;
    const int G = dual_components(REG);
    const double normL2 = first_order(REG) ? 8.0 : 32.0;
    const int64_t N = (int64_t)n1 * n2;
    int st;
    // no column with d_i > 0: P = I exactly
    if (pc && pc->priv && ((const nys_precond_priv*)pc->priv)->ell_eff == 0) pc = nullptr;
    if (pc) {
        // two launches per TV dual step, three per HS one (prox_fused.cu),
        // where the layout allows
        st = prox_dual_fused(ctx, pc, REG, lb, n_inner, sizeof(T) == 8 ? NYS_F64 : NYS_F32, n1, n2, s, out, Q);
        if (st != NYS_EINVAL) return st;
    }
    T* work = (T*)scratch(ctx, SLOT_PROX, prox_work_elems(G, N) * sizeof(T), &st);
    if (st) return st;
    cudaStream_t sm = ctx->stream;
    const int grid = (int)std::min<int64_t>((N + 255) / 256, ctx->sm_count * 8);
    const int dt = sizeof(T) == 8 ? NYS_F64 : NYS_F32;
    const TC step = (TC)(1.0 / (lb * normL2));
    double t = 1.0;
    if (!pc && REG == NYS_REG_TV) {
        // one launch per dual step: x ping-pongs between X[0] and X[1], (R, Q)
        // as in the preconditioned fused step (warm start from Q itself, the
        // last step writes Q unless it reads it)
        T* X[2] = {work, work + N};
        T* RQ[2][2] = {{work + 2 * N, work + 2 * N + G * N}, {work + 2 * N + 2 * G * N, work + 2 * N + 3 * G * N}};
        NYS_CK(ctx, launch_pdl(lt_kernel<T, REG>, grid, 256, 0, sm, Q, s, (TC)lb, n1, n2, n_inner ? X[0] : out,
                               DualStop{}));
        NYS_LAUNCH_CK(ctx);
        for (int k = 0; k < n_inner; ++k) {
            const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
            const double beta = (t - 1.0) / tn;
            t = tn;
            const bool fin = k + 1 == n_inner;
            TvDual<T> d;
            d.x = X[k & 1];
            d.Ro = k ? RQ[k & 1][0] : Q;
            d.Qo = k ? RQ[k & 1][1] : Q;
            d.Rn = fin ? nullptr : RQ[(k + 1) & 1][0];
            d.Qn = (fin && k) ? Q : RQ[(k + 1) & 1][1];
            d.step = step;
            d.beta = (TC)beta;
            DualStop ds;
            if (ctx->dual_stop) ds.flags = ctx->counters + COUNTER_DUAL_STOP;
            ds.k = k;
            NYS_CK(ctx, launch_pdl(tv_dual_x_kernel<T>, grid, 256, 0, sm, d, s, (TC)lb, n1, n2,
                                   fin ? out : X[(k + 1) & 1], ds));
            NYS_LAUNCH_CK(ctx);
        }
        if (n_inner == 1) NYS_CK(ctx, cudaMemcpyAsync(Q, RQ[1][1], sizeof(T) * G * N, cudaMemcpyDeviceToDevice, sm));
        return NYS_OK;
    }
    T* R = work;
    T* Qp = R + G * N;
    T* x = Qp + G * N;
    T* g = x + N;
    NYS_CK(ctx, cudaMemcpyAsync(R, Q, sizeof(T) * G * N, cudaMemcpyDeviceToDevice, sm));
    NYS_CK(ctx, cudaMemcpyAsync(Qp, Q, sizeof(T) * G * N, cudaMemcpyDeviceToDevice, sm));
    for (int k = 0; k < n_inner; ++k) {
        // the exact early stop (internal.cuh): dual_update keeps the flags;
        // the x of a skipped step is not recomputed (P = I)
        DualStop ds;
        if (ctx->dual_stop) ds.flags = ctx->counters + COUNTER_DUAL_STOP;
        ds.k = k;
        if (pc) {
            NYS_CK(ctx, launch_pdl(lt_kernel<T, REG>, grid, 256, 0, sm, R, nullptr, TC(0), n1, n2, g, DualStop{}));
            NYS_LAUNCH_CK(ctx);
            if ((st = precond_run(ctx, pc, 1, dt, g, g, 1))) return st;
            NYS_CK(ctx, launch_pdl(axpy_kernel<T>, grid, 256, 0, sm, s, g, (TC)lb, N, x));
        } else {
            NYS_CK(ctx, launch_pdl(lt_kernel<T, REG>, grid, 256, 0, sm, R, s, (TC)lb, n1, n2, x, ds));
        }
        NYS_LAUNCH_CK(ctx);
        const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        const double beta = (t - 1.0) / tn;
        t = tn;
        NYS_CK(ctx, launch_pdl(dual_update_kernel<T, REG>, grid, 256, 0, sm, x, R, Qp, step, (TC)beta, n1, n2, ds));
        NYS_LAUNCH_CK(ctx);
    }
    // Q_io <- last Q; out = s - lb P^{-1} L^T Q
    NYS_CK(ctx, cudaMemcpyAsync(Q, Qp, sizeof(T) * G * N, cudaMemcpyDeviceToDevice, sm));
    if (pc) {
        NYS_CK(ctx, launch_pdl(lt_kernel<T, REG>, grid, 256, 0, sm, Qp, nullptr, TC(0), n1, n2, g, DualStop{}));
        NYS_LAUNCH_CK(ctx);
        if ((st = precond_run(ctx, pc, 1, dt, g, g, 1))) return st;
        NYS_CK(ctx, launch_pdl(axpy_kernel<T>, grid, 256, 0, sm, s, g, (TC)lb, N, out));
    } else {
        NYS_CK(ctx, launch_pdl(lt_kernel<T, REG>, grid, 256, 0, sm, Qp, s, (TC)lb, n1, n2, out, DualStop{}));
    }
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

// ------------------------------------------------------- wavelet SSN ----
constexpr int SCH = 128;     // pixels per evaluation block
constexpr int SMAXL = 128;   // largest sketch size of the Newton solver

struct SsnState {
    double nF;        // ||F|| at the accepted gamma
    double a;         // current step fraction
    double scale;     // 1 + ||Ubar^T s||
    int done;         // 1 = finished
    int first;        // 1 = no accepted point yet
    int tries;        // step halvings at the current Newton step
    int newton;       // Newton steps taken
    int converged;
};

template <class T>
__device__ __forceinline__ T soft(T z, T tau) {
    const T a = fabs(z) - tau;
    return a > T(0) ? copysign(a, z) : T(0);
}

// Evaluation at gamma_trial: partial F, partial J (upper triangle, float),
// partial Ubar^T s.  Ubar[j][i] = sqrtd[j] * U[j][i].
template <class T>
__global__ void __launch_bounds__(256) ssn_eval_kernel(const T* __restrict__ U, const double* __restrict__ sqd,
                                                       const T* __restrict__ s, int64_t N, int ell, double tau,
                                                       const double* __restrict__ gtrial,
                                                       const SsnState* __restrict__ state, double* __restrict__ Fp,
                                                       double* __restrict__ Sp, float* __restrict__ Jp) {
    pdl_enter();
    if (state->done) return;
    // dynamic shared memory: rr, ss (SCH doubles each), gs, sd (ell doubles
    // each), then the masked Ubar chunk ub (ell x (SCH + 1) floats)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* rr = reinterpret_cast<double*>(smem_raw);
    double* ss = rr + SCH;
    double* gs = ss + SCH;
    double* sd = gs + ell;
    float* ubf = reinterpret_cast<float*>(sd + ell);
    auto ub = [&](int j, int t) -> float& { return ubf[(size_t)j * (SCH + 1) + t]; };
    const int64_t i0 = (int64_t)blockIdx.x * SCH;
    const int cnt = (int)(N - i0 < (int64_t)SCH ? N - i0 : (int64_t)SCH);
    for (int j = threadIdx.x; j < ell; j += blockDim.x) gs[j] = gtrial[j], sd[j] = sqd[j];
    __syncthreads();
    // z = s - Ubar gamma per pixel (one thread per pixel of the chunk)
    for (int t = threadIdx.x; t < SCH; t += blockDim.x) {
        double r = 0.0, sv = 0.0;
        bool m = false;
        if (t < cnt) {
            sv = (double)s[i0 + t];
            double z = sv;
            for (int j = 0; j < ell; ++j) z -= sd[j] * (double)U[(size_t)j * N + i0 + t] * gs[j];
            r = sv - soft(z, tau);
            m = fabs(z) > tau;
        }
        rr[t] = r;
        ss[t] = sv;
        for (int j = 0; j < ell; ++j)
            ub(j, t) = (m && t < cnt) ? (float)(sd[j] * (double)U[(size_t)j * N + i0 + t]) : 0.0f;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double* Fb = Fp + (size_t)blockIdx.x * ell;
    double* Sb = Sp + (size_t)blockIdx.x * ell;
    for (int j = warp; j < ell; j += nw) {
        double f = 0.0, sv = 0.0;
        for (int t = lane; t < cnt; t += 32) {
            const double u = sd[j] * (double)U[(size_t)j * N + i0 + t];
            f += u * rr[t];
            sv += u * ss[t];
        }
        f = warp_sum(f);
        sv = warp_sum(sv);
        if (lane == 0) Fb[j] = f, Sb[j] = sv;
    }
    float* Jb = Jp + (size_t)blockIdx.x * ell * ell;
    for (int e = threadIdx.x; e < ell * ell; e += blockDim.x) {
        const int j = e / ell, k = e - j * ell;
        if (k < j) continue;
        float acc = 0.0f;
        for (int t = 0; t < cnt; ++t) acc = fmaf(ub(j, t), ub(k, t), acc);
        Jb[e] = acc;
    }
}

// One CTA: reduce partials at gamma_trial and run the accept / halve logic.
__global__ void __launch_bounds__(1024) ssn_step_kernel(int nb, int ell, double tol, int max_newton,
                                                        const double* __restrict__ Fp, const double* __restrict__ Sp,
                                                        const float* __restrict__ Jp, double* __restrict__ gamma,
                                                        double* __restrict__ gtrial, double* __restrict__ dir,
                                                        double* __restrict__ Fcur, double* __restrict__ Jw,
                                                        SsnState* __restrict__ st) {
    pdl_enter();
    if (st->done) return;
    __shared__ double F[SMAXL];
    __shared__ double sh[32];
    __shared__ int flag;
    __shared__ int accept;
    for (int j = threadIdx.x; j < ell; j += blockDim.x) {
        double f = 0.0, sv = 0.0;
        for (int b = 0; b < nb; ++b) f += Fp[(size_t)b * ell + j], sv += Sp[(size_t)b * ell + j];
        F[j] = f + gtrial[j];
        if (st->first) Fcur[j] = sv;   // stash Ubar^T s for the scale below
    }
    __syncthreads();
    double n2 = 0.0;
    for (int j = threadIdx.x; j < ell; j += blockDim.x) n2 += F[j] * F[j];
    n2 = block_sum(n2, sh);
    const double nF = sqrt(n2);
    if (threadIdx.x == 0) {
        if (st->first) {
            double s2 = 0.0;
            for (int j = 0; j < ell; ++j) s2 += Fcur[j] * Fcur[j];
            st->scale = 1.0 + sqrt(s2);
        }
        // accept when first, improved, or after the 11th trial of this step
        accept = st->first || nF < st->nF || st->tries >= 10;
    }
    __syncthreads();
    if (!accept) {
        if (threadIdx.x == 0) {
            st->tries += 1;
            st->a *= 0.5;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < ell; j += blockDim.x) gtrial[j] = gamma[j] + st->a * dir[j];
        return;
    }
    // accepted: gamma <- trial, J <- I + sum of partials
    for (int j = threadIdx.x; j < ell; j += blockDim.x) gamma[j] = gtrial[j], Fcur[j] = F[j];
    for (int e = threadIdx.x; e < ell * ell; e += blockDim.x) {
        const int j = e / ell, k = e - j * ell;
        const int a = min(j, k), b = max(j, k);
        double v = 0.0;
        for (int q = 0; q < nb; ++q) v += (double)Jp[(size_t)q * ell * ell + (size_t)a * ell + b];
        Jw[e] = v + (j == k ? 1.0 : 0.0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!st->first) st->newton += 1;
        st->first = 0;
        st->nF = nF;
        st->tries = 0;
        st->a = 1.0;
        if (nF <= tol * st->scale) st->done = 1, st->converged = 1;
        else if (st->newton >= max_newton) st->done = 1;
    }
    __syncthreads();
    if (st->done) return;
    // Newton direction: J d = -F (Cholesky, forward and back substitution)
    const bool ok = block_cholesky(Jw, ell, &flag);
    if (!ok) {
        if (threadIdx.x == 0) st->done = 1;
        return;
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < ell; ++i) {
            double v = -F[i];
            for (int k = 0; k < i; ++k) v -= Jw[(size_t)i * ell + k] * dir[k];
            dir[i] = v / Jw[(size_t)i * ell + i];
        }
        for (int i = ell - 1; i >= 0; --i) {
            double v = dir[i];
            for (int k = i + 1; k < ell; ++k) v -= Jw[(size_t)k * ell + i] * dir[k];
            dir[i] = v / Jw[(size_t)i * ell + i];
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < ell; j += blockDim.x) gtrial[j] = gamma[j] + dir[j];
}

template <class T>
__global__ void ssn_final_kernel(const T* __restrict__ U, const double* __restrict__ sqd, const T* __restrict__ s,
                                 int64_t N, int ell, double tau, const double* __restrict__ gamma, T* __restrict__ out) {
    pdl_enter();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double z = (double)s[i];
        for (int j = 0; j < ell; ++j) z -= sqd[j] * (double)U[(size_t)j * N + i] * gamma[j];
        out[i] = (T)soft(z, tau);
    }
}

template <class T>
__global__ void soft_kernel(const T* __restrict__ s, int64_t N, double tau, T* __restrict__ out) {
    pdl_enter();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (T)soft((double)s[i], tau);
}

__global__ void ssn_init_kernel(SsnState* st, const double* gamma_in, double* gamma, double* gtrial, int ell) {
    pdl_enter();
    for (int j = threadIdx.x; j < ell; j += blockDim.x) {
        const double g = gamma_in ? gamma_in[j] : 0.0;
        gamma[j] = g;
        gtrial[j] = g;
    }
    if (threadIdx.x == 0) {
        st->nF = 0.0;
        st->a = 1.0;
        st->scale = 1.0;
        st->done = 0;
        st->first = 1;
        st->tries = 0;
        st->newton = 0;
        st->converged = 0;
    }
}

}  // namespace

// Semi-smooth Newton prox; `max_evals` evaluation/step pairs are launched
// (later ones exit at once when done).  If `sync_until_done`, the host keeps
// launching batches until the device reports completion.
template <class T>
int ssn_run(nys_ctx* ctx, const nys_precond* pc, double tau, int64_t N, const T* s, T* out, double* gamma_io,
            int max_newton, int evals_per_batch, bool sync_until_done, nys_prox_info* info) {
    const int ell = pc->ell;
    if (ell > SMAXL) return fail(ctx, NYS_EINVAL, "prox_wavelet: sketch size above %d is not supported", SMAXL);
    const auto* pv = (const nys_precond_priv*)pc->priv;
    const int nb = (int)((N + SCH - 1) / SCH);
    int st;
    const size_t need = sizeof(SsnState) + 64 + (size_t)(6 * ell + ell * ell) * 8 + (size_t)nb * ell * 16 +
                        (size_t)nb * ell * ell * 4;
    char* w = (char*)scratch(ctx, SLOT_SSN, need, &st);
    if (st) return st;
    SsnState* state = (SsnState*)w;
    double* gamma = (double*)(w + ((sizeof(SsnState) + 63) & ~size_t(63)));
    double* gtrial = gamma + ell;
    double* dir = gtrial + ell;
    double* Fcur = dir + ell;
    double* Jw = Fcur + ell;
    double* Fp = Jw + (size_t)ell * ell;
    double* Sp = Fp + (size_t)nb * ell;
    float* Jp = (float*)(Sp + (size_t)nb * ell);
    cudaStream_t sm = ctx->stream;
    const double tol = sizeof(T) == 8 ? 1e-12 : 1e-6;
    NYS_CK(ctx, launch_pdl(ssn_init_kernel, 1, 256, 0, sm, state, (const double*)gamma_io, gamma, gtrial, ell));
    NYS_LAUNCH_CK(ctx);
    const T* U = (const T*)pc->U;
    const size_t esm = (size_t)(2 * SCH + 2 * ell) * sizeof(double) + (size_t)ell * (SCH + 1) * sizeof(float);
    if (int st2 = smem_optin(ctx, (const void*)ssn_eval_kernel<T>, esm)) return st2;
    int launched = 0;
    const int max_evals = max_newton * 12 + 1;
    while (true) {
        for (int e = 0; e < evals_per_batch; ++e) {
            NYS_CK(ctx, launch_pdl(ssn_eval_kernel<T>, nb, 256, esm, sm, U, (const double*)pv->sqrtd, s, N, ell, tau,
                                   (const double*)gtrial, (const SsnState*)state, Fp, Sp, Jp));
            NYS_LAUNCH_CK(ctx);
            NYS_CK(ctx, launch_pdl(ssn_step_kernel, 1, 1024, 0, sm, nb, ell, tol, max_newton, (const double*)Fp,
                                   (const double*)Sp, (const float*)Jp, gamma, gtrial, dir, Fcur, Jw, state));
            NYS_LAUNCH_CK(ctx);
        }
        launched += evals_per_batch;
        if (!sync_until_done) break;
        SsnState h;
        NYS_CK(ctx, cudaMemcpyAsync(&h, state, sizeof(h), cudaMemcpyDeviceToHost, sm));
        NYS_CK(ctx, cudaStreamSynchronize(sm));
        if (h.done || launched >= max_evals) break;
    }
    const int grid = (int)std::min<int64_t>((N + 255) / 256, ctx->sm_count * 8);
    NYS_CK(ctx, launch_pdl(ssn_final_kernel<T>, grid, 256, 0, sm, U, (const double*)pv->sqrtd, s, N, ell, tau,
                           (const double*)gamma, out));
    NYS_LAUNCH_CK(ctx);
    if (gamma_io) NYS_CK(ctx, cudaMemcpyAsync(gamma_io, gamma, ell * sizeof(double), cudaMemcpyDeviceToDevice, sm));
    if (info) {
        SsnState h;
        NYS_CK(ctx, cudaMemcpyAsync(&h, state, sizeof(h), cudaMemcpyDeviceToHost, sm));
        NYS_CK(ctx, cudaStreamSynchronize(sm));
        info->iterations = h.newton;
        info->converged = h.converged;
        info->residual = h.nF;
    }
    return NYS_OK;
}

template int ssn_run<float>(nys_ctx*, const nys_precond*, double, int64_t, const float*, float*, double*, int, int,
                            bool, nys_prox_info*);
template int ssn_run<double>(nys_ctx*, const nys_precond*, double, int64_t, const double*, double*, double*, int, int,
                             bool, nys_prox_info*);

template <class T>
int soft_run(nys_ctx* ctx, double tau, int64_t N, const T* s, T* out) {
    const int grid = (int)std::min<int64_t>((N + 255) / 256, ctx->sm_count * 8);
    NYS_CK(ctx, launch_pdl(soft_kernel<T>, grid, 256, 0, ctx->stream, s, N, tau, out));
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}
template int soft_run<float>(nys_ctx*, double, int64_t, const float*, float*);
template int soft_run<double>(nys_ctx*, double, int64_t, const double*, double*);

int prox_dual_run(nys_ctx* ctx, const nys_precond* pc, int reg, double lb, int n_inner, int dtype, int n1, int n2,
                  const void* s, void* out, void* Q) {
    auto go = [&](auto* tag) -> int {
        using T = std::remove_pointer_t<decltype(tag)>;
        const T* sp = (const T*)s;
        T* op = (T*)out;
        T* qp = (T*)Q;
        switch (reg) {
            case NYS_REG_TV: return prox_dual_typed<T, NYS_REG_TV>(ctx, pc, lb, n_inner, n1, n2, sp, op, qp);
            case NYS_REG_ISOTV: return prox_dual_typed<T, NYS_REG_ISOTV>(ctx, pc, lb, n_inner, n1, n2, sp, op, qp);
            case NYS_REG_HS: return prox_dual_typed<T, NYS_REG_HS>(ctx, pc, lb, n_inner, n1, n2, sp, op, qp);
            case NYS_REG_HS2: return prox_dual_typed<T, NYS_REG_HS2>(ctx, pc, lb, n_inner, n1, n2, sp, op, qp);
            case NYS_REG_HSINF: return prox_dual_typed<T, NYS_REG_HSINF>(ctx, pc, lb, n_inner, n1, n2, sp, op, qp);
        }
        return fail(ctx, NYS_EINVAL, "prox: regulariser %d has no dual prox", reg);
    };
    return dtype == NYS_F64 ? go((double*)nullptr) : go((float*)nullptr);
}

}  // namespace nys

using namespace nys;

extern "C" {

static int check_prox(nys_ctx* ctx, const nys_precond* pc, int dtype, int64_t N, const void* s, const void* out) {
    if (!ctx || !s || !out) return fail(ctx, NYS_EINVAL, "prox: null argument");
    if (dtype != NYS_F32 && dtype != NYS_F64) return fail(ctx, NYS_EINVAL, "prox: dtype must be f32 or f64");
    if (pc) {
        if (!pc->priv) return fail(ctx, NYS_EINVAL, "prox: preconditioner not factored");
        if (pc->N != N) return fail(ctx, NYS_EINVAL, "prox: preconditioner size %lld != %lld", (long long)pc->N,
                                    (long long)N);
        if (pc->mu != pc->mu) return fail(ctx, NYS_EINVAL, "prox: call nys_precond_setup first");
    }
    return NYS_OK;
}

int prox_tv(nys_ctx* ctx, const nys_precond* pc, double lb, int n_inner, int dtype, int n1, int n2, const void* s,
            void* out, void* Q) {
    if (int st = check_prox(ctx, pc, dtype, (int64_t)n1 * n2, s, out)) return st;
    if (!Q || n1 <= 0 || n2 <= 0 || n_inner < 0 || !(lb > 0.0)) return fail(ctx, NYS_EINVAL, "prox_tv: bad argument");
    return prox_dual_run(ctx, pc, NYS_REG_TV, lb, n_inner, dtype, n1, n2, s, out, Q);
}

int prox_hs(nys_ctx* ctx, const nys_precond* pc, double lb, int n_inner, int dtype, int n1, int n2, const void* s,
            void* out, void* Q) {
    if (int st = check_prox(ctx, pc, dtype, (int64_t)n1 * n2, s, out)) return st;
    if (!Q || n1 <= 0 || n2 <= 0 || n_inner < 0 || !(lb > 0.0)) return fail(ctx, NYS_EINVAL, "prox_hs: bad argument");
    return prox_dual_run(ctx, pc, NYS_REG_HS, lb, n_inner, dtype, n1, n2, s, out, Q);
}

int prox_mixed(nys_ctx* ctx, const nys_precond* pc, int reg, double lb, int n_inner, int dtype, int n1, int n2,
               const void* s, void* out, void* Q) {
    if (int st = check_prox(ctx, pc, dtype, (int64_t)n1 * n2, s, out)) return st;
    if (!Q || n1 <= 0 || n2 <= 0 || n_inner < 0 || !(lb > 0.0))
        return fail(ctx, NYS_EINVAL, "prox_mixed: bad argument");
    if (reg != NYS_REG_TV && reg != NYS_REG_ISOTV && reg != NYS_REG_HS && reg != NYS_REG_HS2 && reg != NYS_REG_HSINF)
        return fail(ctx, NYS_EINVAL, "prox_mixed: regulariser %d has no dual prox", reg);
    return prox_dual_run(ctx, pc, reg, lb, n_inner, dtype, n1, n2, s, out, Q);
}

int prox_wavelet(nys_ctx* ctx, const nys_precond* pc, double tau, int dtype, int64_t N, const void* s, void* out,
                 double* gamma_io, nys_prox_info* info) {
    if (int st = check_prox(ctx, pc, dtype, N, s, out)) return st;
    if (!(tau >= 0.0)) return fail(ctx, NYS_EINVAL, "prox_wavelet: tau must be >= 0");
    if (!pc) {
        if (info) info->iterations = 0, info->converged = 1, info->residual = 0.0;
        return dtype == NYS_F64 ? soft_run<double>(ctx, tau, N, (const double*)s, (double*)out)
                                : soft_run<float>(ctx, tau, N, (const float*)s, (float*)out);
    }
    if ((pc->dtype == NYS_F64) != (dtype == NYS_F64) || pc->dtype == NYS_BF16)
        return fail(ctx, NYS_EINVAL, "prox_wavelet: factor dtype must match the data (f32 or f64)");
    if (dtype == NYS_F64)
        return ssn_run<double>(ctx, pc, tau, N, (const double*)s, (double*)out, gamma_io, 50, 4, true, info);
    return ssn_run<float>(ctx, pc, tau, N, (const float*)s, (float*)out, gamma_io, 50, 4, true, info);
}

}  // extern "C"
