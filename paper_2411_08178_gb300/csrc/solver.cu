// Weighted accelerated proximal gradient, Algorithm 3, for
//     min_x f(x) + lambda g(x),   f = 1/2 ||A x - y||^2  or  sum huber_delta(A x - y),
// with g = anisotropic TV, Hessian Schatten-1, or ||xbar||_1 of the Haar
// coefficients xbar = W x (invertible-L form, Sec. III-B).  Per iteration:
//     grad = A^T A u - A^T y            (one fused normal-operator pass), or
//            A^T clip(A u - y, +-delta) (Huber), or W (A^T A W^T u) - W A^T y
//     s    = u - alpha P^{-1} grad
//     x'   = prox^P_{alpha lambda g}(s)  (dual APG / semi-smooth Newton)
//     t'   = (1 + sqrt(1 + 4 t^2))/2,  u = x' + ((t - 1)/t') (x' - x)
// x^1 = u^1 = 0, t^0 = 1.  alpha defaults to 1/(1.02 lambda_max(P^{-1} Phi)),
// lambda_max from 50 power-iteration steps from a seeded Gaussian start.
//
// Launch structure: one iteration is a fixed sequence of kernels (the momentum
// scalar t lives on the device, double-buffered by iteration parity, and the
// two iterate buffers swap roles every iteration), so the solver captures the
// even and the odd iteration once into CUDA graphs on its own stream and
// replays them: one graph launch per iteration instead of ~60 kernel launches.
#include "internal.cuh"

#include <cmath>

namespace nys {
template <class T>
int ssn_run(nys_ctx* ctx, const nys_precond* pc, double tau, int64_t N, const T* s, T* out, double* gamma_io,
            int max_newton, int evals_per_batch, bool sync_until_done, nys_prox_info* info);
template <class T>
int soft_run(nys_ctx* ctx, double tau, int64_t N, const T* s, T* out);
int prox_dual_run(nys_ctx* ctx, const nys_precond* pc, int reg, double lb, int n_inner, int dtype, int n1, int n2,
                  const void* s, void* out, void* Q);
}  // namespace nys

struct nys_solver {
    nys_ctx* ctx = nullptr;
    nys_op* op = nullptr;
    nys_solver_desc d{};
    const nys_precond* pc = nullptr;
    int dt = NYS_F32;
    int64_t N = 0, M = 0;
    int G = 0;
    void* mem = nullptr;
    // buffers (op dtype); X[parity] is the current iterate
    void *y = nullptr, *aty = nullptr, *u = nullptr, *s = nullptr, *g = nullptr;
    void* X[2] = {nullptr, nullptr};
    void *tM = nullptr, *tN = nullptr, *Q = nullptr;
    double* gamma = nullptr;
    double* pw = nullptr;     // [0] power-iteration norm, [2], [3]: t slots by parity
    double* npart = nullptr;  // per-CTA partial sums of the power-iteration norm
    double alpha = 0.0;
    int parity = 0;
    int k = 0;
    // graph replay
    cudaStream_t gs = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int64_t glaunch[2] = {0, 0};
    bool gvalid = false;
    uint64_t gen = 0;   // ctx->scratch_gen when the graphs were captured
};

namespace nys {
namespace {

template <class T>
__global__ void sub_kernel(T* __restrict__ a, const T* __restrict__ b, int64_t n) {
    pdl_enter();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = a[i] - b[i];
}

template <class T>
__global__ void huber_resid_kernel(T* __restrict__ r, const T* __restrict__ y, int64_t n, double delta) {
    pdl_enter();
    using TC = typename Comp<T>::type;
    const TC d = (TC)delta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = (T)fmin(d, fmax(-d, (TC)r[i] - (TC)y[i]));
}

// s = u - alpha * g
template <class T>
__global__ void step_kernel(const T* __restrict__ u, const T* __restrict__ g, double alpha, int64_t n,
                            T* __restrict__ s) {
    pdl_enter();
    using TC = typename Comp<T>::type;
    const TC a = (TC)alpha;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s[i] = (T)((TC)u[i] - a * (TC)g[i]);
}

// t' = (1 + sqrt(1 + 4 t^2))/2 from t_in; u = xn + ((t - 1)/t') (xn - x);
// t' written to t_out by one thread (t_in and t_out are different slots)
template <class T>
__global__ void momentum_kernel(const T* __restrict__ xn, const T* __restrict__ x, const double* __restrict__ t_in,
                                double* __restrict__ t_out, int64_t n, T* __restrict__ u) {
    pdl_enter();
    using TC = typename Comp<T>::type;
    const double t = *t_in;
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    const TC b = (TC)((t - 1.0) / tn);
    if (blockIdx.x == 0 && threadIdx.x == 0) *t_out = tn;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const TC a = (TC)xn[i];
        u[i] = (T)(a + b * (a - (TC)x[i]));
    }
}

// power iteration helpers: part[b] = block b's share of ||w||^2, then every
// CTA sums the partials in the same order, w /= ||w|| and out[0] = ||w||
template <class T>
__global__ void __launch_bounds__(256) sumsq_part_kernel(const T* __restrict__ w, int64_t n, double* __restrict__ part) {
    pdl_enter();
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)w[i];
        s += v * v;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <class T>
__global__ void __launch_bounds__(256) scale_by_norm_kernel(T* __restrict__ w, int64_t n,
                                                            const double* __restrict__ part, int np,
                                                            double* __restrict__ out) {
    pdl_enter();
    __shared__ double sh[32];
    double s = 0.0;
    for (int t = threadIdx.x; t < np; t += blockDim.x) s += part[t];
    s = block_sum(s, sh);
    const double nr = sqrt(s);
    if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = nr;
    const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = (T)((double)w[i] * inv);
}

// Gaussian start vector of the power iteration: splitmix64 (Steele, Lea and
// Flood, OOPSLA 2014) hashes of (seed, i) turned into N(0,1) by Box-Muller
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class T>
__global__ void gauss_init_kernel(T* __restrict__ w, int64_t n, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t a = splitmix64(seed ^ splitmix64(2 * (uint64_t)i));
        const uint64_t b = splitmix64(seed ^ splitmix64(2 * (uint64_t)i + 1));
        const double u0 = ((double)(a >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u1 = ((double)(b >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        w[i] = (T)(sqrt(-2.0 * log(u0)) * cospi(2.0 * u1));
    }
}

__global__ void set_t_kernel(double* t) {
    t[0] = 1.0;
    t[1] = 1.0;
}

// ------------------------------------------------------------ objective --
// part[2 b]   = sum of the data term over the block's entries of r = A x - y
// part[2 b+1] = sum of the regulariser over the block's pixels
template <class T, int REG>
__global__ void objective_kernel(const T* __restrict__ r, const T* __restrict__ y, int64_t M, int fit, double delta,
                                 const T* __restrict__ x, int n1, int n2, double* __restrict__ part) {
    __shared__ double sh[32];
    double f = 0.0, g = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < M; t += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)r[t] - (double)y[t];
        const double a = fabs(v);
        f += (fit == NYS_FIT_HUBER && a > delta) ? delta * a - 0.5 * delta * delta : 0.5 * v * v;
    }
    const int64_t N = (int64_t)n1 * n2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / n2), j = (int)(t - (int64_t)i * n2);
        auto X = [&](int a, int b) { return (double)x[(size_t)pmod(a, n1) * n2 + pmod(b, n2)]; };
        if (REG == NYS_REG_TV || REG == NYS_REG_ISOTV) {
            const double g1 = X(i, j) - X(i - 1, j), g2 = X(i, j) - X(i, j - 1);
            g += REG == NYS_REG_TV ? fabs(g1) + fabs(g2) : sqrt(g1 * g1 + g2 * g2);
        } else if (REG == NYS_REG_HS || REG == NYS_REG_HS2 || REG == NYS_REG_HSINF) {
            const double v11 = X(i - 1, j) - 2.0 * X(i, j) + X(i + 1, j);
            const double v22 = X(i, j - 1) - 2.0 * X(i, j) + X(i, j + 1);
            const double v12 = 0.25 * (X(i + 1, j + 1) - X(i + 1, j - 1) - X(i - 1, j + 1) + X(i - 1, j - 1));
            const double m = 0.5 * (v11 + v22), h = 0.5 * (v11 - v22);
            const double rr = sqrt(h * h + v12 * v12);
            // Schatten-1, -2 (Frobenius, cross term twice) or -inf of [[v11, v12], [v12, v22]]
            g += REG == NYS_REG_HS ? fabs(m + rr) + fabs(m - rr)
                 : REG == NYS_REG_HS2 ? sqrt(v11 * v11 + 2.0 * v12 * v12 + v22 * v22)
                                      : fabs(m) + rr;
        } else {
            g += fabs((double)x[t]);
        }
    }
    f = block_sum(f, sh);
    g = block_sum(g, sh);
    if (threadIdx.x == 0) part[2 * blockIdx.x] = f, part[2 * blockIdx.x + 1] = g;
}

__global__ void objective_sum_kernel(const double* __restrict__ part, int nb, double lambda,
                                     double* __restrict__ out) {
    __shared__ double sh[32];
    double f = 0.0, g = 0.0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) f += part[2 * t], g += part[2 * t + 1];
    f = block_sum(f, sh);
    g = block_sum(g, sh);
    if (threadIdx.x == 0) out[0] = f + lambda * g, out[1] = f, out[2] = g;
}

inline int grid_for(nys_ctx* ctx, int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, ctx->sm_count * 8); }

template <class T>
int phi_apply(nys_solver* S, const void* v, void* out) {
    // Phi = A^T A, or W A^T A W^T for the wavelet model
    nys_op* op = S->op;
    if (S->d.reg != NYS_REG_WAVELET) return op_run(op, 2, v, out, 1, S->dt, S->dt);
    int st;
    if ((st = haar_run(op, v, S->tN, 1, 1, S->dt, S->dt))) return st;
    if ((st = op_run(op, 2, S->tN, S->s, 1, S->dt, S->dt))) return st;
    return haar_run(op, S->s, out, 1, 0, S->dt, S->dt);
}

template <class T>
int gradient(nys_solver* S) {
    nys_ctx* ctx = S->ctx;
    nys_op* op = S->op;
    const int dt = S->dt;
    int st;
    const int gN = grid_for(ctx, S->N), gM = grid_for(ctx, S->M);
    if (S->d.reg == NYS_REG_WAVELET) {
        // g = W A^T A W^T u - W A^T y
        if ((st = haar_run(op, S->u, S->tN, 1, 1, dt, dt))) return st;
        if (S->d.fit == NYS_FIT_HUBER) {
            if ((st = op_run(op, 0, S->tN, S->tM, 1, dt, dt))) return st;
            NYS_CK(ctx, launch_pdl(huber_resid_kernel<T>, gM, 256, 0, ctx->stream, (T*)S->tM, (const T*)S->y, S->M,
                               S->d.huber_delta));
            NYS_LAUNCH_CK(ctx);
            if ((st = op_run(op, 1, S->tM, S->s, 1, dt, dt))) return st;
            return haar_run(op, S->s, S->g, 1, 0, dt, dt);
        }
        if ((st = op_run(op, 2, S->tN, S->s, 1, dt, dt))) return st;
        if ((st = haar_run(op, S->s, S->g, 1, 0, dt, dt))) return st;
        NYS_CK(ctx, launch_pdl(sub_kernel<T>, gN, 256, 0, ctx->stream, (T*)S->g, (const T*)S->aty, S->N));
        NYS_LAUNCH_CK(ctx);
        return NYS_OK;
    }
    if (S->d.fit == NYS_FIT_HUBER) {
        if ((st = op_run(op, 0, S->u, S->tM, 1, dt, dt))) return st;
        NYS_CK(ctx, launch_pdl(huber_resid_kernel<T>, gM, 256, 0, ctx->stream, (T*)S->tM, (const T*)S->y, S->M,
                               S->d.huber_delta));
        NYS_LAUNCH_CK(ctx);
        return op_run(op, 1, S->tM, S->g, 1, dt, dt);
    }
    if ((st = op_run(op, 2, S->u, S->g, 1, dt, dt))) return st;
    NYS_CK(ctx, launch_pdl(sub_kernel<T>, gN, 256, 0, ctx->stream, (T*)S->g, (const T*)S->aty, S->N));
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

// one iteration of Algorithm 3 with the given parity, issued on ctx->stream
template <class T>
int iterate_one(nys_solver* S, int par) {
    nys_ctx* ctx = S->ctx;
    const int gN = grid_for(ctx, S->N);
    void* x = S->X[par];
    void* xn = S->X[par ^ 1];
    int st;
    if ((st = gradient<T>(S))) return st;
    if (S->pc && (st = precond_run(ctx, S->pc, 1, S->dt, S->g, S->g, 1))) return st;
    NYS_CK(ctx, launch_pdl(step_kernel<T>, gN, 256, 0, ctx->stream, (const T*)S->u, (const T*)S->g, S->alpha, S->N,
                           (T*)S->s));
    NYS_LAUNCH_CK(ctx);
    const double tau = S->alpha * S->d.lambda;
    if (S->d.reg == NYS_REG_WAVELET) {
        if (S->pc) st = ssn_run<T>(ctx, S->pc, tau, S->N, (const T*)S->s, (T*)xn, S->gamma, 50, 10, false, nullptr);
        else st = soft_run<T>(ctx, tau, S->N, (const T*)S->s, (T*)xn);
    } else {
        st = prox_dual_run(ctx, S->pc, S->d.reg, tau, S->d.n_inner, S->dt, S->op->n1, S->op->n2, S->s, xn, S->Q);
    }
    if (st) return st;
    NYS_CK(ctx, launch_pdl(momentum_kernel<T>, gN, 256, 0, ctx->stream, (const T*)xn, (const T*)x, S->pw + 2 + par,
                           S->pw + 2 + (par ^ 1), S->N, (T*)S->u));
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

template <class T>
int capture(nys_solver* S) {
    nys_ctx* ctx = S->ctx;
    cudaStream_t saved = ctx->stream;
    // the captured kernels carry the context's L2 access-policy window
    cudaStreamAttrValue v = {};
    if (ctx->l2_window_set) v = ctx->l2_window;
    NYS_CK(ctx, cudaStreamSetAttribute(S->gs, cudaStreamAttributeAccessPolicyWindow, &v));
    for (int par = 0; par < 2; ++par) {
        if (S->gexec[par]) {
            cudaGraphExecDestroy(S->gexec[par]);
            S->gexec[par] = nullptr;
        }
        const int64_t l0 = ctx->launches;
        ctx->stream = S->gs;
        NYS_CK(ctx, cudaStreamBeginCapture(S->gs, cudaStreamCaptureModeRelaxed));
        int st = iterate_one<T>(S, par);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(S->gs, &graph);
        ctx->stream = saved;
        if (st) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
        const cudaError_t ei = cudaGraphInstantiate(&S->gexec[par], graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return cuda_fail(ctx, ei, "cudaGraphInstantiate");
        S->glaunch[par] = ctx->launches - l0;
        ctx->launches = l0;
    }
    S->gvalid = true;
    S->gen = ctx->scratch_gen;
    return NYS_OK;
}

template <class T>
int iterate(nys_solver* S, int n_steps) {
    nys_ctx* ctx = S->ctx;
    int st;
    if (S->d.no_graph) {
        for (int it = 0; it < n_steps; ++it) {
            if ((st = iterate_one<T>(S, S->parity))) return st;
            S->parity ^= 1;
            S->k += 1;
        }
        return NYS_OK;
    }
    // the graphs hold the addresses of the context's scratch regions: if any
    // was reallocated since (by another object on this context), capture again
    if (S->gen != ctx->scratch_gen) S->gvalid = false;
    if (!S->gvalid && (st = capture<T>(S))) return st;
    NYS_CK(ctx, cudaEventRecord(S->ev_in, ctx->stream));
    NYS_CK(ctx, cudaStreamWaitEvent(S->gs, S->ev_in, 0));
    for (int it = 0; it < n_steps; ++it) {
        NYS_CK(ctx, cudaGraphLaunch(S->gexec[S->parity], S->gs));
        ctx->launches += S->glaunch[S->parity];
        S->parity ^= 1;
        S->k += 1;
    }
    NYS_CK(ctx, cudaEventRecord(S->ev_out, S->gs));
    NYS_CK(ctx, cudaStreamWaitEvent(ctx->stream, S->ev_out, 0));
    return NYS_OK;
}

template <class T>
int estimate_alpha(nys_solver* S) {
    nys_ctx* ctx = S->ctx;
    cudaStream_t s = ctx->stream;
    T* z = (T*)S->X[1];   // scratch vectors before the first iteration
    T* w = (T*)S->u;
    gauss_init_kernel<T><<<grid_for(ctx, S->N), 256, 0, s>>>(z, S->N, S->d.power_seed);
    NYS_LAUNCH_CK(ctx);
    const int gN = grid_for(ctx, S->N);
    auto normalise = [&](T* v) -> int {
        NYS_CK(ctx, launch_pdl(sumsq_part_kernel<T>, gN, 256, 0, s, v, S->N, S->npart));
        NYS_LAUNCH_CK(ctx);
        NYS_CK(ctx, launch_pdl(scale_by_norm_kernel<T>, gN, 256, 0, s, v, S->N, (const double*)S->npart, gN, S->pw));
        NYS_LAUNCH_CK(ctx);
        return NYS_OK;
    };
    int st;
    if ((st = normalise(z))) return st;
    const int iters = S->d.power_iters > 0 ? S->d.power_iters : 50;
    for (int it = 0; it < iters; ++it) {
        if ((st = phi_apply<T>(S, z, w))) return st;
        if (S->pc && (st = precond_run(ctx, S->pc, 1, S->dt, w, w, 1))) return st;
        if ((st = normalise(w))) return st;
        std::swap(z, w);
    }
    double lam = 0.0;
    NYS_CK(ctx, cudaMemcpyAsync(&lam, S->pw, sizeof(double), cudaMemcpyDeviceToHost, s));
    NYS_CK(ctx, cudaStreamSynchronize(s));
    if (!(lam > 0.0) || !std::isfinite(lam)) return fail(ctx, NYS_ENONFINITE, "power iteration gave %g", lam);
    const double a = 1.0 / (1.02 * lam);
    if (a != S->alpha) S->gvalid = false;   // alpha is baked into the captured graphs
    S->alpha = a;
    return NYS_OK;
}

template <class T>
int reset_state(nys_solver* S) {
    cudaStream_t s = S->ctx->stream;
    const size_t nb = S->N * sizeof(T);
    NYS_CK(S->ctx, cudaMemsetAsync(S->X[0], 0, nb, s));
    NYS_CK(S->ctx, cudaMemsetAsync(S->X[1], 0, nb, s));
    NYS_CK(S->ctx, cudaMemsetAsync(S->u, 0, nb, s));
    if (S->G) NYS_CK(S->ctx, cudaMemsetAsync(S->Q, 0, (size_t)S->G * nb, s));
    if (S->gamma && S->pc) NYS_CK(S->ctx, cudaMemsetAsync(S->gamma, 0, S->pc->ell * sizeof(double), s));
    set_t_kernel<<<1, 1, 0, s>>>(S->pw + 2);
    NYS_LAUNCH_CK(S->ctx);
    S->parity = 0;
    S->k = 0;
    return NYS_OK;
}

template <class T>
int load_data(nys_solver* S, const void* y) {
    nys_ctx* ctx = S->ctx;
    const size_t es = sizeof(T);
    NYS_CK(ctx, cudaMemcpyAsync(S->y, y, S->M * es, cudaMemcpyDeviceToDevice, ctx->stream));
    int st;
    // A^T y (and W A^T y for the wavelet model)
    if ((st = op_run(S->op, 1, S->y, S->aty, 1, S->dt, S->dt))) return st;
    if (S->d.reg == NYS_REG_WAVELET) {
        if ((st = haar_run(S->op, S->aty, S->tN, 1, 0, S->dt, S->dt))) return st;
        NYS_CK(ctx, cudaMemcpyAsync(S->aty, S->tN, S->N * es, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return NYS_OK;
}

template <class T>
int create_typed(nys_solver* S, const void* y) {
    nys_ctx* ctx = S->ctx;
    const int64_t N = S->N, M = S->M;
    const size_t es = sizeof(T);
    const int ell = S->pc ? S->pc->ell : 0;
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    const size_t total = al(M * es) * 2 + al(N * es) * 7 + al((size_t)S->G * N * es) + al((ell + 1) * 8) + 256 +
                         al((size_t)ctx->sm_count * 8 * sizeof(double));
    NYS_CK(ctx, cudaMalloc(&S->mem, total));
    char* p = (char*)S->mem;
    auto take = [&](size_t n) {
        char* r = p;
        p += al(n);
        return r;
    };
    S->y = take(M * es);
    S->tM = take(M * es);
    S->aty = take(N * es);
    S->X[0] = take(N * es);
    S->X[1] = take(N * es);
    S->u = take(N * es);
    S->s = take(N * es);
    S->g = take(N * es);
    S->tN = take(N * es);
    S->Q = S->G ? take((size_t)S->G * N * es) : nullptr;
    S->gamma = (double*)take((ell + 1) * 8);
    S->pw = (double*)take(256);
    S->npart = (double*)take((size_t)ctx->sm_count * 8 * sizeof(double));
    NYS_CK(ctx, cudaStreamCreateWithFlags(&S->gs, cudaStreamNonBlocking));
    NYS_CK(ctx, cudaEventCreateWithFlags(&S->ev_in, cudaEventDisableTiming));
    NYS_CK(ctx, cudaEventCreateWithFlags(&S->ev_out, cudaEventDisableTiming));
    int st;
    if ((st = load_data<T>(S, y))) return st;
    if ((st = reset_state<T>(S))) return st;
    if (S->d.alpha > 0.0) S->alpha = S->d.alpha;
    else if ((st = estimate_alpha<T>(S))) return st;
    if ((st = reset_state<T>(S))) return st;
    // reserve the scratch that pgd_step uses, so later steps never allocate
    if (S->G) {
        if (!scratch(ctx, SLOT_PROX, prox_work_elems(S->G, N) * es, &st)) return st;
    }
    if (S->pc) {
        // the largest of the P^{-1} / prox partial-sum layouts (chunks of 1024 or
        // 2048 pixels)
        const size_t nbp = (size_t)((N + 511) / 512);   // chunks of 512 .. 2048 pixels
        if (!scratch(ctx, SLOT_PRECOND, (nbp * ell + 2 * ell) * es, &st)) return st;
        if (S->d.reg == NYS_REG_WAVELET) {
            // the first ssn_run call sizes SLOT_SSN; run one prox now
            if ((st = ssn_run<T>(ctx, S->pc, 0.0, N, (const T*)S->X[0], (T*)S->X[1], nullptr, 1, 1, false, nullptr)))
                return st;
            if ((st = reset_state<T>(S))) return st;
        }
    }
    if (S->op->haar_levels > 0 && !scratch(ctx, SLOT_OPTMP, 2 * (size_t)N * es, &st)) return st;
    return NYS_OK;
}

}  // namespace
}  // namespace nys

using namespace nys;

extern "C" {

int nys_solver_create(nys_ctx* ctx, nys_op* op, const nys_solver_desc* d, const void* y, const nys_precond* pc,
                      nys_solver** out) {
    if (!ctx || !op || !d || !y || !out) return fail(ctx, NYS_EINVAL, "nys_solver_create: null argument");
    if (d->reg != NYS_REG_WAVELET && d->reg != NYS_REG_TV && d->reg != NYS_REG_HS && d->reg != NYS_REG_ISOTV &&
        d->reg != NYS_REG_HS2 && d->reg != NYS_REG_HSINF)
        return fail(ctx, NYS_EINVAL, "nys_solver_create: unknown regulariser");
    if (d->reg == NYS_REG_WAVELET && op->haar_levels <= 0)
        return fail(ctx, NYS_EINVAL, "nys_solver_create: the wavelet model needs haar_levels > 0");
    if (d->fit != NYS_FIT_L2 && d->fit != NYS_FIT_HUBER) return fail(ctx, NYS_EINVAL, "nys_solver_create: fit");
    if (!(d->lambda >= 0.0)) return fail(ctx, NYS_EINVAL, "nys_solver_create: lambda must be >= 0");
    if (d->reg != NYS_REG_WAVELET && d->n_inner <= 0) return fail(ctx, NYS_EINVAL, "nys_solver_create: n_inner");
    if (pc) {
        if (!pc->priv || pc->N != op->N) return fail(ctx, NYS_EINVAL, "nys_solver_create: preconditioner mismatch");
        if (pc->mu != pc->mu) return fail(ctx, NYS_EINVAL, "nys_solver_create: call nys_precond_setup first");
    }
    auto* S = new nys_solver();
    S->ctx = ctx;
    ctx_retain(ctx);
    S->op = op;
    S->d = *d;
    S->pc = pc;
    S->dt = op->dtype;
    S->N = op->N;
    S->M = op->M;
    S->G = d->reg == NYS_REG_WAVELET ? 0 : (d->reg == NYS_REG_TV || d->reg == NYS_REG_ISOTV ? 2 : 3);
    const int st = S->dt == NYS_F64 ? create_typed<double>(S, y) : create_typed<float>(S, y);
    if (st) {
        nys_solver_destroy(S);
        return st;
    }
    *out = S;
    return NYS_OK;
}

int nys_solver_destroy(nys_solver* S) {
    if (!S) return NYS_OK;
    cudaStreamSynchronize(S->ctx->stream);
    if (S->gs) cudaStreamSynchronize(S->gs);
    for (auto& g : S->gexec)
        if (g) cudaGraphExecDestroy(g);
    if (S->ev_in) cudaEventDestroy(S->ev_in);
    if (S->ev_out) cudaEventDestroy(S->ev_out);
    if (S->gs) cudaStreamDestroy(S->gs);
    if (S->mem) cudaFree(S->mem);
    nys_ctx* ctx = S->ctx;
    delete S;
    ctx_release(ctx);
    return NYS_OK;
}

int pgd_step(nys_solver* S, int n_steps) {
    if (!S) return fail(nullptr, NYS_EINVAL, "pgd_step: null solver");
    if (n_steps < 0) return fail(S->ctx, NYS_EINVAL, "pgd_step: negative step count");
    if (n_steps == 0) return NYS_OK;
    return S->dt == NYS_F64 ? iterate<double>(S, n_steps) : iterate<float>(S, n_steps);
}

int nys_solver_reset(nys_solver* S) {
    if (!S) return fail(nullptr, NYS_EINVAL, "null solver");
    return S->dt == NYS_F64 ? reset_state<double>(S) : reset_state<float>(S);
}

int nys_solver_set_data(nys_solver* S, const void* y) {
    if (!S || !y) return fail(S ? S->ctx : nullptr, NYS_EINVAL, "nys_solver_set_data: null argument");
    int st = S->dt == NYS_F64 ? load_data<double>(S, y) : load_data<float>(S, y);
    if (st) return st;
    return S->dt == NYS_F64 ? reset_state<double>(S) : reset_state<float>(S);
}

int nys_solver_restart(nys_solver* S, int reestimate_alpha) {
    if (!S) return fail(nullptr, NYS_EINVAL, "null solver");
    int st;
    if (reestimate_alpha && S->d.alpha <= 0.0) {
        if (S->pc && S->pc->mu != S->pc->mu) return fail(S->ctx, NYS_EINVAL, "restart: preconditioner not set up");
        st = S->dt == NYS_F64 ? estimate_alpha<double>(S) : estimate_alpha<float>(S);
        if (st) return st;
    }
    return S->dt == NYS_F64 ? reset_state<double>(S) : reset_state<float>(S);
}

int nys_solver_get_x(nys_solver* S, void* x_out) {
    if (!S || !x_out) return fail(S ? S->ctx : nullptr, NYS_EINVAL, "nys_solver_get_x: null argument");
    void* x = S->X[S->parity];
    if (S->d.reg == NYS_REG_WAVELET) return haar_run(S->op, x, x_out, 1, 1, S->dt, S->dt);
    NYS_CK(S->ctx, cudaMemcpyAsync(x_out, x, S->N * dtype_size(S->dt), cudaMemcpyDeviceToDevice, S->ctx->stream));
    return NYS_OK;
}

int nys_solver_objective(nys_solver* S, double* F) {
    if (!S || !F) return fail(S ? S->ctx : nullptr, NYS_EINVAL, "nys_solver_objective: null argument");
    nys_ctx* ctx = S->ctx;
    cudaStream_t s = ctx->stream;
    const void* x = S->X[S->parity];
    int st;
    // r = A x (image domain: W^T xbar for the wavelet model), into tM
    const void* img = x;
    if (S->d.reg == NYS_REG_WAVELET) {
        if ((st = haar_run(S->op, x, S->tN, 1, 1, S->dt, S->dt))) return st;
        img = S->tN;
    }
    if ((st = op_run(S->op, 0, img, S->tM, 1, S->dt, S->dt))) return st;
    const int nb = std::max(1, std::min<int>(ctx->sm_count * 2, (int)((std::max(S->M, S->N) + 255) / 256)));
    double* buf = (double*)scratch(ctx, SLOT_MISC, (size_t)(2 * nb + 4) * sizeof(double), &st);
    if (st) return st;
    double* out = buf;
    double* part = buf + 4;
    auto launch = [&](auto* tag) -> int {
        using T = std::remove_pointer_t<decltype(tag)>;
        const T* r = (const T*)S->tM;
        const T* yy = (const T*)S->y;
        const T* xx = (const T*)x;
        auto k = objective_kernel<T, NYS_REG_WAVELET>;
        switch (S->d.reg) {
            case NYS_REG_TV: k = objective_kernel<T, NYS_REG_TV>; break;
            case NYS_REG_ISOTV: k = objective_kernel<T, NYS_REG_ISOTV>; break;
            case NYS_REG_HS: k = objective_kernel<T, NYS_REG_HS>; break;
            case NYS_REG_HS2: k = objective_kernel<T, NYS_REG_HS2>; break;
            case NYS_REG_HSINF: k = objective_kernel<T, NYS_REG_HSINF>; break;
        }
        k<<<nb, 256, 0, s>>>(r, yy, S->M, S->d.fit, S->d.huber_delta, xx, S->op->n1, S->op->n2, part);
        NYS_LAUNCH_CK(ctx);
        return NYS_OK;
    };
    if ((st = S->dt == NYS_F64 ? launch((double*)nullptr) : launch((float*)nullptr))) return st;
    objective_sum_kernel<<<1, 256, 0, s>>>(part, nb, S->d.lambda, out);
    NYS_LAUNCH_CK(ctx);
    double h[3];
    NYS_CK(ctx, cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
    NYS_CK(ctx, cudaStreamSynchronize(s));
    F[0] = h[0];
    return NYS_OK;
}

int nys_solver_alpha(nys_solver* S, double* alpha) {
    if (!S || !alpha) return fail(nullptr, NYS_EINVAL, "nys_solver_alpha: null argument");
    *alpha = S->alpha;
    return NYS_OK;
}

}  // extern "C"
