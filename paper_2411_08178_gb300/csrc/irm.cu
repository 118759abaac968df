// Iteratively reweighted minimisation (Algorithm 2) for the l_p - l_q problem
// of Eq. lplqReg with L the first differences, its x-step solved by
// preconditioned conjugate gradients with the Nystrom preconditioner of
// Phi_k built on the fly every outer iteration (Sec. III-A).
//
// Outer iteration k, from x = x^{k-1}:
//   W_f = |A x - y|_eps^{p-2}, W_g = |L x|_eps^{q-2}          (Eqs. v:z:updating, WfWg:IRM)
//   b   = A^T W_f y,  Phi_k = A^T W_f A + lambda L^T W_g L   (Eq. lplq:sub:updateX:linearEq)
//   ell > 0: Omega (seed + k), Y = Phi_k Omega, Algorithm 1, P^{-1} (mu = 0)
//   x   = PCG(Phi_k, b) started from x^{k-1}
// |r|_eps = sqrt(r^2 + eps).  Every vector is in the operator's dtype; the
// sketch is stored in store_dtype (bf16 or float32 for float32 operators).
// CG scalars stay on the device (fixed-order float64 reductions); the host
// reads ||r||^2 once per CG iteration for the stopping test.
#include "internal.cuh"
#include "stencil.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace nys {
namespace {

enum { S_RZ = 0, S_ALPHA = 1, S_BETA = 2, S_RR = 3, S_COUNT = 8 };

template <class T>
__global__ void irm_data_weights(const T* __restrict__ Ax, const T* __restrict__ y, int64_t M,
                                 typename Comp<T>::type e, typename Comp<T>::type eps, T* __restrict__ wf,
                                 T* __restrict__ wfy) {
    pdl_enter();
    using TC = typename Comp<T>::type;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
        const TC yv = (TC)y[m];
        const TC r = (TC)Ax[m] - yv;
        const TC w = pow(r * r + eps, e);
        wf[m] = (T)w;
        wfy[m] = (T)(w * yv);
    }
}

// both components of L x = (x - x(up), x - x(left)) at every pixel
template <class T>
__global__ void irm_grad_weights(const T* __restrict__ x, int n1, int n2, typename Comp<T>::type e,
                                 typename Comp<T>::type eps, T* __restrict__ wg) {
    pdl_enter();
    using TC = typename Comp<T>::type;
    const int64_t N = (int64_t)n1 * n2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        int i, j;
        pix_ij(t, n2, i, j);
        const TC xc = (TC)x[t];
        const TC g1 = xc - (TC)x[(size_t)wrap_dec(i, n1) * n2 + j];
        const TC g2 = xc - (TC)x[(size_t)i * n2 + wrap_dec(j, n2)];
        wg[t] = (T)pow(g1 * g1 + eps, e);
        wg[N + t] = (T)pow(g2 * g2 + eps, e);
    }
}

// v[b][m] *= w[m]
template <class TV, class TW>
__global__ void irm_scale(TV* __restrict__ v, const TW* __restrict__ w, int64_t M, int nb) {
    pdl_enter();
    const int64_t total = (int64_t)nb * M;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
        v[t] = (TV)((TW)v[t] * w[t % M]);
}

// out[b] += lam L^T (W_g L u[b]) with L the first differences:
// (L^T v)(i,j) = v1(i,j) - v1(i+1,j) + v2(i,j) - v2(i,j+1), v = W_g L u
template <class TI, class TO, class TW>
__global__ void irm_wlap_add(const TI* __restrict__ u, TO* __restrict__ out, const TW* __restrict__ wg, TW lam,
                             int n1, int n2, int nb) {
    pdl_enter();
    const int64_t N = (int64_t)n1 * n2;
    const int64_t total = (int64_t)nb * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / N, pix = t - b * N;
        int i, j;
        pix_ij(pix, n2, i, j);
        const TI* ub = u + b * N;
        const size_t r0 = (size_t)i * n2, rm = (size_t)wrap_dec(i, n1) * n2, rp = (size_t)wrap_inc(i, n1) * n2;
        const int jm = wrap_dec(j, n2), jp = wrap_inc(j, n2);
        const TW c = (TW)ldf(ub + r0 + j);
        const TW v1 = wg[r0 + j] * (c - (TW)ldf(ub + rm + j));
        const TW v1d = wg[rp + j] * ((TW)ldf(ub + rp + j) - c);
        const TW v2 = wg[N + r0 + j] * (c - (TW)ldf(ub + r0 + jm));
        const TW v2r = wg[N + r0 + jp] * ((TW)ldf(ub + r0 + jp) - c);
        stf(out + t, (TW)ldf(out + t) + lam * ((v1 - v1d) + (v2 - v2r)));
    }
}

template <class T>
__global__ void __launch_bounds__(256) irm_dot_part(const T* __restrict__ a, const T* __restrict__ b, int64_t n,
                                                   double* __restrict__ part) {
    pdl_enter();
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        s += (double)a[t] * (double)b[t];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// sum of the partials in a fixed order, then: mode 0 rr = s; 1 alpha = rz / s;
// 2 beta = s / rz, rz = s; 3 rz = s
__global__ void __launch_bounds__(256) irm_dot_fin(const double* __restrict__ part, int np, int mode,
                                                  double* __restrict__ sc) {
    pdl_enter();
    __shared__ double sh[32];
    double s = 0.0;
    for (int t = threadIdx.x; t < np; t += blockDim.x) s += part[t];
    s = block_sum(s, sh);
    if (threadIdx.x != 0) return;
    if (mode == 0) sc[S_RR] = s;
    else if (mode == 1) sc[S_ALPHA] = sc[S_RZ] / s;
    else if (mode == 2) sc[S_BETA] = s / sc[S_RZ], sc[S_RZ] = s;
    else sc[S_RZ] = s;
}

template <class T>
__global__ void irm_cg_xr(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ q,
                          int64_t n, const double* __restrict__ sc) {
    pdl_enter();
    using TC = typename Comp<T>::type;
    const TC a = (TC)sc[S_ALPHA];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        x[t] = (T)((TC)x[t] + a * (TC)p[t]);
        r[t] = (T)((TC)r[t] - a * (TC)q[t]);
    }
}

template <class T>
__global__ void irm_cg_p(T* __restrict__ p, const T* __restrict__ z, int64_t n, const double* __restrict__ sc) {
    pdl_enter();
    using TC = typename Comp<T>::type;
    const TC be = (TC)sc[S_BETA];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        p[t] = (T)((TC)z[t] + be * (TC)p[t]);
}

// r = b - r
template <class T>
__global__ void irm_rsub(const T* __restrict__ b, T* __restrict__ r, int64_t n) {
    pdl_enter();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        r[t] = b[t] - r[t];
}

}  // namespace
}  // namespace nys

struct nys_irm {
    nys_ctx* ctx = nullptr;
    nys_op* op = nullptr;
    nys_irm_desc d = {};
    int dt = NYS_F32;
    int64_t N = 0, M = 0;
    void *y = nullptr, *x = nullptr, *xp = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr,
         *b = nullptr, *tM = nullptr, *wf = nullptr, *wfy = nullptr, *wg = nullptr;
    double* sc = nullptr;      // device scalars
    double* part = nullptr;    // reduction partials
    double* host_rr = nullptr; // pinned
    int np = 0;
    // on-the-fly preconditioner
    void *Om = nullptr, *Y = nullptr, *tB = nullptr;
    int chunk = 0;
    nys_precond pc = {};
    int k = 0;
    std::vector<void*> owned;
};

namespace nys {
namespace {

template <class T>
struct Irm {
    using TC = typename Comp<T>::type;
    nys_irm* S;
    nys_ctx* ctx;
    cudaStream_t s;
    int grid;
    explicit Irm(nys_irm* s_) : S(s_), ctx(s_->ctx), s(s_->ctx->stream) {
        grid = (int)std::min<int64_t>((std::max(S->N, S->M) + 255) / 256, (int64_t)ctx->sm_count * 8);
    }
    int dot(const void* a, const void* b, int64_t n, int mode) {
        NYS_CK(ctx, launch_pdl(irm_dot_part<T>, S->np, 256, 0, s, (const T*)a, (const T*)b, n, S->part));
        NYS_LAUNCH_CK(ctx);
        NYS_CK(ctx, launch_pdl(irm_dot_fin, 1, 256, 0, s, (const double*)S->part, S->np, mode, S->sc));
        NYS_LAUNCH_CK(ctx);
        return NYS_OK;
    }
    // the last mode-0 reduction, on the host (synchronises the stream)
    int read_rr(double* out) {
        NYS_CK(ctx, cudaMemcpyAsync(S->host_rr, S->sc + S_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
        NYS_CK(ctx, cudaStreamSynchronize(s));
        *out = *S->host_rr;
        return NYS_OK;
    }
    // out = Phi_k u = A^T W_f A u + lambda L^T W_g L u
    int phi(const void* u, void* out) {
        int st;
        nys_op* op = S->op;
        if ((st = op_run(op, 0, u, S->tM, 1, S->dt, S->dt))) return st;
        NYS_CK(ctx, launch_pdl(irm_scale<T, T>, grid, 256, 0, s, (T*)S->tM, (const T*)S->wf, S->M, 1));
        NYS_LAUNCH_CK(ctx);
        if ((st = op_run(op, 1, S->tM, out, 1, S->dt, S->dt))) return st;
        NYS_CK(ctx, launch_pdl(irm_wlap_add<T, T, T>, grid, 256, 0, s, (const T*)u, (T*)out, (const T*)S->wg,
                               (T)S->d.lambda, op->n1, op->n2, 1));
        NYS_LAUNCH_CK(ctx);
        return NYS_OK;
    }
    // Y = Phi_k Omega for the ell probe images, in chunks through tB
    template <class TS>
    int sketch(int ell) {
        int st;
        nys_op* op = S->op;
        const int sdt = S->d.store_dtype;
        if ((st = omega_fill(ctx, sdt, S->Om, (int64_t)ell * S->N, S->d.seed + (uint64_t)S->k))) return st;
        for (int b0 = 0; b0 < ell; b0 += S->chunk) {
            const int nb = std::min(S->chunk, ell - b0);
            const TS* om = (const TS*)S->Om + (size_t)b0 * S->N;
            TS* yy = (TS*)S->Y + (size_t)b0 * S->N;
            if ((st = op_run(op, 0, om, S->tB, nb, sdt, S->dt))) return st;
            NYS_CK(ctx, launch_pdl(irm_scale<T, T>, grid, 256, 0, s, (T*)S->tB, (const T*)S->wf, S->M, nb));
            NYS_LAUNCH_CK(ctx);
            if ((st = op_run(op, 1, S->tB, yy, nb, S->dt, sdt))) return st;
            NYS_CK(ctx, launch_pdl(irm_wlap_add<TS, TS, T>, grid, 256, 0, s, om, yy, (const T*)S->wg, (T)S->d.lambda,
                                   op->n1, op->n2, nb));
            NYS_LAUNCH_CK(ctx);
        }
        const double eps_mach = S->dt == NYS_F64 ? std::ldexp(1.0, -52) : std::ldexp(1.0, -23);
        if ((st = nys_factor(ctx, S->Om, S->Y, sdt, S->N, ell, eps_mach, &S->pc))) return st;
        return nys_precond_setup(ctx, &S->pc, 0.0, 0);
    }
    int step(nys_irm_info* info) {
        int st;
        nys_op* op = S->op;
        const int64_t N = S->N;
        const TC ep = (TC)(0.5 * (S->d.p - 2.0)), eq = (TC)(0.5 * (S->d.q - 2.0)), eps = (TC)S->d.eps;
        // weights at x^{k-1}
        if ((st = op_run(op, 0, S->x, S->tM, 1, S->dt, S->dt))) return st;
        NYS_CK(ctx, launch_pdl(irm_data_weights<T>, grid, 256, 0, s, (const T*)S->tM, (const T*)S->y, S->M, ep, eps,
                               (T*)S->wf, (T*)S->wfy));
        NYS_LAUNCH_CK(ctx);
        NYS_CK(ctx, launch_pdl(irm_grad_weights<T>, grid, 256, 0, s, (const T*)S->x, op->n1, op->n2, eq, eps,
                               (T*)S->wg));
        NYS_LAUNCH_CK(ctx);
        if ((st = op_run(op, 1, S->wfy, S->b, 1, S->dt, S->dt))) return st;
        const bool pre = S->d.ell > 0;
        if (pre) {
            st = S->d.store_dtype == NYS_BF16 ? sketch<__nv_bfloat16>(S->d.ell)
                 : S->d.store_dtype == NYS_F64 ? sketch<double>(S->d.ell) : sketch<float>(S->d.ell);
            if (st) return st;
        }
        NYS_CK(ctx, cudaMemcpyAsync(S->xp, S->x, N * sizeof(T), cudaMemcpyDeviceToDevice, s));
        double v;
        if ((st = dot(S->b, S->b, N, 0)) || (st = read_rr(&v))) return st;
        const double nb = std::sqrt(v);
        // r = b - Phi x, z = P^{-1} r, p = z
        if ((st = phi(S->x, S->r))) return st;
        NYS_CK(ctx, launch_pdl(irm_rsub<T>, grid, 256, 0, s, (const T*)S->b, (T*)S->r, N));
        NYS_LAUNCH_CK(ctx);
        if ((st = dot(S->r, S->r, N, 0)) || (st = read_rr(&v))) return st;
        double rn = std::sqrt(v);
        int it = 0;
        if (rn > S->d.cg_tol * nb) {
            auto precond = [&]() -> int {
                if (pre) return precond_run(ctx, &S->pc, 1, S->dt, S->r, S->z, 1);
                NYS_CK(ctx, cudaMemcpyAsync(S->z, S->r, N * sizeof(T), cudaMemcpyDeviceToDevice, s));
                return NYS_OK;
            };
            if ((st = precond())) return st;
            NYS_CK(ctx, cudaMemcpyAsync(S->p, S->z, N * sizeof(T), cudaMemcpyDeviceToDevice, s));
            if ((st = dot(S->r, S->z, N, 3))) return st;
            while (it < S->d.cg_max) {
                ++it;
                if ((st = phi(S->p, S->q))) return st;
                if ((st = dot(S->p, S->q, N, 1))) return st;
                NYS_CK(ctx, launch_pdl(irm_cg_xr<T>, grid, 256, 0, s, (T*)S->x, (T*)S->r, (const T*)S->p,
                                       (const T*)S->q, N, (const double*)S->sc));
                NYS_LAUNCH_CK(ctx);
                if ((st = dot(S->r, S->r, N, 0)) || (st = read_rr(&v))) return st;
                rn = std::sqrt(v);
                if (!(rn > S->d.cg_tol * nb)) break;
                if ((st = precond())) return st;
                if ((st = dot(S->r, S->z, N, 2))) return st;
                NYS_CK(ctx, launch_pdl(irm_cg_p<T>, grid, 256, 0, s, (T*)S->p, (const T*)S->z, N,
                                       (const double*)S->sc));
                NYS_LAUNCH_CK(ctx);
            }
        }
        // ||x^k - x^{k-1}|| / ||x^k||
        NYS_CK(ctx, launch_pdl(irm_rsub<T>, grid, 256, 0, s, (const T*)S->x, (T*)S->xp, N));   // xp = x - xp
        NYS_LAUNCH_CK(ctx);
        if ((st = dot(S->xp, S->xp, N, 0)) || (st = read_rr(&v))) return st;
        const double dx = std::sqrt(v);
        if ((st = dot(S->x, S->x, N, 0)) || (st = read_rr(&v))) return st;
        const double nx = std::sqrt(v);
        S->k += 1;
        if (info) {
            info->cg_iters = it;
            info->residual = nb > 0.0 ? rn / nb : 0.0;
            info->rel_change = nx > 0.0 ? dx / nx : 0.0;
        }
        return NYS_OK;
    }
};

void irm_free(nys_irm* S) {
    if (!S) return;
    if (S->ctx) cudaStreamSynchronize(S->ctx->stream);
    for (void* p : S->owned) cudaFree(p);
    if (S->host_rr) cudaFreeHost(S->host_rr);
    if (S->pc.priv) nys_precond_release(&S->pc);
    if (S->ctx) ctx_release(S->ctx);
    delete S;
}

}  // namespace
}  // namespace nys

using namespace nys;

extern "C" {

int nys_irm_create(nys_ctx* ctx, nys_op* op, const nys_irm_desc* d, const void* y, nys_irm** out) {
    if (!ctx || !op || !d || !y || !out) return fail(ctx, NYS_EINVAL, "nys_irm_create: null argument");
    if (!(d->p > 0.0 && d->p <= 2.0) || !(d->q > 0.0 && d->q <= 2.0) || !(d->eps > 0.0) || !(d->lambda >= 0.0) ||
        d->ell < 0 || d->cg_max < 1 || !(d->cg_tol > 0.0))
        return fail(ctx, NYS_EINVAL, "nys_irm_create: need 0 < p, q <= 2, eps > 0, lambda >= 0, cg_max >= 1");
    const bool f64 = op->dtype == NYS_F64;
    if (d->ell > 0 && (f64 ? d->store_dtype != NYS_F64 : (d->store_dtype != NYS_F32 && d->store_dtype != NYS_BF16)))
        return fail(ctx, NYS_EINVAL, "nys_irm_create: store dtype does not match the operator");
    if (d->ell > 1024 || d->ell > op->N) return fail(ctx, NYS_EINVAL, "nys_irm_create: ell above min(N, 1024)");
    auto* S = new nys_irm();
    S->ctx = ctx;
    ctx_retain(ctx);
    S->op = op;
    S->d = *d;
    S->dt = op->dtype;
    S->N = op->N;
    S->M = op->M;
    const size_t es = dtype_size(S->dt);
    auto take = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(bytes, 256)) != cudaSuccess) return nullptr;
        S->owned.push_back(p);
        return p;
    };
    const size_t nN = (size_t)S->N * es, nM = (size_t)S->M * es;
    S->y = take(nM);
    S->x = take(nN);
    S->xp = take(nN);
    S->r = take(nN);
    S->z = take(nN);
    S->p = take(nN);
    S->q = take(nN);
    S->b = take(nN);
    S->tM = take(nM);
    S->wf = take(nM);
    S->wfy = take(nM);
    S->wg = take(2 * nN);
    S->np = ctx->sm_count * 2;
    S->part = (double*)take((size_t)S->np * sizeof(double));
    S->sc = (double*)take(S_COUNT * sizeof(double));
    bool ok = S->y && S->x && S->xp && S->r && S->z && S->p && S->q && S->b && S->tM && S->wf && S->wfy && S->wg &&
              S->part && S->sc && cudaMallocHost(&S->host_rr, sizeof(double)) == cudaSuccess;
    if (ok && d->ell > 0) {
        const size_t ss = dtype_size(d->store_dtype);
        S->chunk = std::min(d->ell, 32);
        S->Om = take((size_t)d->ell * S->N * ss);
        S->Y = take((size_t)d->ell * S->N * ss);
        S->tB = take((size_t)S->chunk * S->M * es);
        void* U = take((size_t)d->ell * S->N * ss);
        void* Sh = take((size_t)d->ell * sizeof(double));
        ok = S->Om && S->Y && S->tB && U && Sh;
        S->pc.U = U;
        S->pc.S_hat = (double*)Sh;
        S->pc.N = S->N;
        S->pc.ell = d->ell;
        S->pc.dtype = d->store_dtype;
    }
    if (!ok) {
        irm_free(S);
        return fail(ctx, NYS_ENOMEM, "nys_irm_create: device allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(S->y, y, nM, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->x, 0, nN, ctx->stream);
    if (e != cudaSuccess) {
        irm_free(S);
        return cuda_fail(ctx, e, "nys_irm_create: copy y");
    }
    *out = S;
    return NYS_OK;
}

int nys_irm_step(nys_irm* S, nys_irm_info* info) {
    if (!S) return fail(nullptr, NYS_EINVAL, "nys_irm_step: null handle");
    if (S->dt == NYS_F64) return Irm<double>(S).step(info);
    return Irm<float>(S).step(info);
}

int nys_irm_get_x(const nys_irm* S, void* x) {
    if (!S || !x) return fail(S ? S->ctx : nullptr, NYS_EINVAL, "nys_irm_get_x: null argument");
    NYS_CK(S->ctx, cudaMemcpyAsync(x, S->x, (size_t)S->N * dtype_size(S->dt), cudaMemcpyDeviceToDevice,
                                   S->ctx->stream));
    return NYS_OK;
}

int nys_irm_reset(nys_irm* S) {
    if (!S) return fail(nullptr, NYS_EINVAL, "nys_irm_reset: null handle");
    NYS_CK(S->ctx, cudaMemsetAsync(S->x, 0, (size_t)S->N * dtype_size(S->dt), S->ctx->stream));
    S->k = 0;
    return NYS_OK;
}

int nys_irm_destroy(nys_irm* S) {
    irm_free(S);
    return NYS_OK;
}

}  // extern "C"
