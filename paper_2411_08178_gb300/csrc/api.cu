// Context, error handling, operator handles and dispatch of the C ABI.
#include "internal.cuh"

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

namespace {
std::mutex g_err_mu;
std::string g_err;
}  // namespace

namespace nys {

void ctx_retain(nys_ctx* ctx) {
    if (ctx) ++ctx->refs;
}

void ctx_release(nys_ctx* ctx) {
    if (!ctx || --ctx->refs > 0) return;
    cudaStreamSynchronize(ctx->stream);
    for (int i = 0; i < 12; ++i)
        if (ctx->slot_ptr[i]) cudaFree(ctx->slot_ptr[i]);
    if (ctx->counters) cudaFree(ctx->counters);
    delete ctx;
}

int fail(nys_ctx* ctx, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    std::lock_guard<std::mutex> g(g_err_mu);
    g_err = buf;
    return code;
}

int cuda_fail(nys_ctx* ctx, cudaError_t e, const char* what) {
    // reset the runtime's last-error state so that a later, unrelated launch
    // check does not report this (non-sticky) error again
    cudaGetLastError();
    return fail(ctx, e == cudaErrorMemoryAllocation ? NYS_ENOMEM : NYS_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

// The dynamic shared-memory opt-in is a property of a kernel on one device:
// remember, per (kernel, device), the largest size granted so far, under a
// lock, so that contexts on several devices (or several host threads) each
// get their own opt-in before their first launch.
int smem_optin(nys_ctx* ctx, const void* func, size_t bytes) {
    if (bytes <= 48 * 1024) return NYS_OK;
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> granted;
    std::lock_guard<std::mutex> g(mu);
    size_t& have = granted[{func, ctx ? ctx->device : 0}];
    if (have >= bytes) return NYS_OK;
    const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute(MaxDynamicSharedMemorySize)");
    have = bytes;
    return NYS_OK;
}

int l2_keep_cols(const nys_ctx* ctx, int64_t N, size_t es, int le) {
    static const double frac = [] {
        const char* e = getenv("NYS_L2_KEEP");
        const double f = e ? atof(e) : 0.5;
        return (f >= 0.0 && f <= 1.0) ? f : 0.5;
    }();
    if (le <= 0 || N <= 0) return 0;
    const double budget = frac * (double)(ctx->l2_bytes > 0 ? ctx->l2_bytes : 0);
    const double per_col = (double)N * (double)es;
    return (int)std::min<double>((double)le, std::floor(budget / per_col));
}

int pdl_mode() {
    static const int m = [] {
        const char* e = getenv("NYS_PDL");
        return (e && e[0] == '0') ? 0 : (e && e[0] == '2') ? 2 : 1;
    }();
    return m;
}

void* scratch(nys_ctx* ctx, int slot, size_t bytes, int* status) {
    *status = NYS_OK;
    if (bytes == 0) bytes = 256;
    if (ctx->slot_bytes[slot] >= bytes) return ctx->slot_ptr[slot];
    // growing is not allowed while the stream is being captured
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        *status = fail(ctx, NYS_ENOMEM, "scratch slot %d needs %zu bytes during stream capture; "
                                        "call once before capturing or nys_reserve()", slot, bytes);
        return nullptr;
    }
    if (ctx->slot_ptr[slot]) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->slot_ptr[slot]);
        ctx->slot_ptr[slot] = nullptr;
        ctx->slot_bytes[slot] = 0;
        ++ctx->scratch_gen;
    }
    size_t nb = (bytes + 4095) & ~size_t(4095);
    cudaError_t e = cudaMalloc(&ctx->slot_ptr[slot], nb);
    if (e != cudaSuccess) {
        ctx->slot_ptr[slot] = nullptr;
        *status = cuda_fail(ctx, e, "scratch cudaMalloc");
        return nullptr;
    }
    ctx->slot_bytes[slot] = nb;
    return ctx->slot_ptr[slot];
}

int op_run(nys_op* op, int which, const void* x, void* y, int batch, int in_dt, int out_dt) {
    switch (op->kind) {
        case NYS_OP_BLUR: return blur_run(op, which, x, y, batch, in_dt, out_dt);
        case NYS_OP_BLUR_DECIM: return decim_run(op, which, x, y, batch, in_dt, out_dt);
        case NYS_OP_RADON: return radon_run(op, which, x, y, batch, in_dt, out_dt);
        case NYS_OP_FANBEAM: return fanbeam_run(op, which, x, y, batch, in_dt, out_dt);
    }
    return fail(op->ctx, NYS_EINVAL, "unknown operator kind %d", op->kind);
}

}  // namespace nys

using namespace nys;

extern "C" {

const char* nys_version(void) { return "nys 0.1 (sm_103a)"; }

int nys_l2_persist(nys_ctx* ctx, const void* ptr, size_t bytes, double hit_ratio) {
    if (!ctx) return fail(nullptr, NYS_EINVAL, "nys_l2_persist: null ctx");
    if (!ctx->stream) return fail(ctx, NYS_EINVAL, "nys_l2_persist: needs a non-default stream");
    cudaStreamAttrValue v = {};
    if (ptr && bytes) {
        int maxp = 0, maxw = 0;
        NYS_CK(ctx, cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, ctx->device));
        NYS_CK(ctx, cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, ctx->device));
        if (maxp <= 0 || maxw <= 0) return fail(ctx, NYS_EINVAL, "nys_l2_persist: not supported on this device");
        NYS_CK(ctx, cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)maxp));
        const size_t win = std::min(bytes, (size_t)maxw);
        v.accessPolicyWindow.base_ptr = const_cast<void*>(ptr);
        v.accessPolicyWindow.num_bytes = win;
        v.accessPolicyWindow.hitRatio = (float)std::min(1.0, std::max(0.0, hit_ratio * (double)maxp / (double)win));
        v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    } else {
        v.accessPolicyWindow.num_bytes = 0;
        v.accessPolicyWindow.hitProp = cudaAccessPropertyNormal;
        v.accessPolicyWindow.missProp = cudaAccessPropertyNormal;
        cudaCtxResetPersistingL2Cache();
    }
    NYS_CK(ctx, cudaStreamSetAttribute(ctx->stream, cudaStreamAttributeAccessPolicyWindow, &v));
    ctx->l2_window = v;
    ctx->l2_window_set = ptr && bytes;
    return NYS_OK;
}

int nys_launch_count(const nys_ctx* ctx, int64_t* count) {
    if (!ctx || !count) return fail(nullptr, NYS_EINVAL, "nys_launch_count: null argument");
    *count = ctx->launches;
    return NYS_OK;
}

int nys_set_dual_stop(nys_ctx* ctx, int on) {
    if (!ctx) return fail(nullptr, NYS_EINVAL, "nys_set_dual_stop: null context");
    ctx->dual_stop = on != 0;
    return NYS_OK;
}

int nys_dual_steps_skipped(nys_ctx* ctx, int64_t* count) {
    if (!ctx || !count) return fail(ctx, NYS_EINVAL, "nys_dual_steps_skipped: null argument");
    unsigned v = 0;
    NYS_CK(ctx, cudaMemcpyAsync(&v, ctx->counters + nys::COUNTER_DUAL_SKIPPED, sizeof(unsigned),
                                cudaMemcpyDeviceToHost, ctx->stream));
    NYS_CK(ctx, cudaStreamSynchronize(ctx->stream));
    *count = v;
    return NYS_OK;
}

const char* nys_last_error(const nys_ctx* ctx) {
    if (ctx) return ctx->err.c_str();
    std::lock_guard<std::mutex> g(g_err_mu);
    static thread_local std::string copy;
    copy = g_err;
    return copy.c_str();
}

int nys_create(nys_ctx** out, int device, void* stream) {
    if (!out) return fail(nullptr, NYS_EINVAL, "nys_create: null output");
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(nullptr, NYS_EINVAL, "nys_create: bad device %d", device);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
    auto* c = new nys_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    {
        int l2 = 0;
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
        c->l2_bytes = l2;
    }
    // completion counters of the last-CTA reductions (zero between launches)
    e = cudaMalloc(&c->counters, COUNTER_WORDS * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->counters, 0, COUNTER_WORDS * sizeof(unsigned));
    if (e != cudaSuccess) {
        if (c->counters) cudaFree(c->counters);
        delete c;
        return cuda_fail(nullptr, e, "nys_create: counters");
    }
    *out = c;
    return NYS_OK;
}

int nys_destroy(nys_ctx* ctx) {
    if (!ctx) return NYS_OK;
    cudaStreamSynchronize(ctx->stream);
    ctx_release(ctx);
    return NYS_OK;
}

int nys_set_stream(nys_ctx* ctx, void* stream) {
    if (!ctx) return fail(nullptr, NYS_EINVAL, "null ctx");
    ctx->stream = (cudaStream_t)stream;
    return NYS_OK;
}

int nys_sync(nys_ctx* ctx) {
    if (!ctx) return fail(nullptr, NYS_EINVAL, "null ctx");
    NYS_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return NYS_OK;
}

int nys_reserve(nys_ctx* ctx, size_t bytes) {
    if (!ctx) return fail(nullptr, NYS_EINVAL, "null ctx");
    int st;
    for (int s = 0; s < SLOT_COUNT; ++s) {
        scratch(ctx, s, bytes, &st);
        if (st) return st;
    }
    return NYS_OK;
}

int nys_op_create(nys_ctx* ctx, const nys_op_desc* d, nys_op** out) {
    if (!ctx || !d || !out) return fail(ctx, NYS_EINVAL, "nys_op_create: null argument");
    if (d->dtype != NYS_F32 && d->dtype != NYS_F64)
        return fail(ctx, NYS_EINVAL, "operator dtype must be NYS_F32 or NYS_F64");
    if (d->n1 <= 0 || d->n2 <= 0) return fail(ctx, NYS_EINVAL, "bad image size %d x %d", d->n1, d->n2);
    auto* op = new nys_op();
    op->ctx = ctx;
    ctx_retain(ctx);
    op->kind = d->kind;
    op->dtype = d->dtype;
    op->n1 = d->n1;
    op->n2 = d->n2;
    op->N = (int64_t)d->n1 * d->n2;
    if (d->n1 <= 0 || d->n2 <= 0 || op->N >= (int64_t(1) << 31)) {
        nys_op_destroy(op);
        return fail(ctx, NYS_EINVAL, "image size must be positive with fewer than 2^31 pixels");
    }
    op->haar_levels = d->haar_levels;
    op->wavelet = d->wavelet;
    if (d->wavelet != NYS_WAVELET_HAAR && d->wavelet != NYS_WAVELET_DB4) {
        nys_op_destroy(op);
        return fail(ctx, NYS_EINVAL, "unknown wavelet %d", d->wavelet);
    }
    if (d->haar_levels < 0 || (d->haar_levels > 0 && ((d->n1 % (1 << d->haar_levels)) ||
                                                     (d->n2 % (1 << d->haar_levels))))) {
        nys_op_destroy(op);
        return fail(ctx, NYS_EINVAL, "image size not divisible by 2^haar_levels");
    }
    int st = NYS_OK;
    if (d->kind == NYS_OP_BLUR || d->kind == NYS_OP_BLUR_DECIM) {
        if (!d->kernel || d->kh <= 0 || d->kw <= 0 || !(d->kh & 1) || !(d->kw & 1)) {
            nys_op_destroy(op);
            return fail(ctx, NYS_EINVAL, "blur kernel must be given with odd sizes");
        }
        op->kh = d->kh;
        op->kw = d->kw;
        op->h.assign(d->kernel, d->kernel + (size_t)d->kh * d->kw);
        op->decim = d->kind == NYS_OP_BLUR_DECIM ? d->decim : 1;
        if (op->decim < 1 || d->n1 % op->decim || d->n2 % op->decim) {
            nys_op_destroy(op);
            return fail(ctx, NYS_EINVAL, "decimation factor must divide the image size");
        }
        op->M = (int64_t)(d->n1 / op->decim) * (d->n2 / op->decim);
        st = blur_setup(op);
    } else if (d->kind == NYS_OP_RADON) {
        if (d->n_angles <= 0 || d->n_bins <= 0 || !(d->angle_span > 0.0) ||
            (int64_t)d->n_angles * d->n_bins >= (int64_t(1) << 31)) {
            nys_op_destroy(op);
            return fail(ctx, NYS_EINVAL, "radon geometry needs n_angles, n_bins > 0, span > 0 and fewer than 2^31 bins");
        }
        op->n_angles = d->n_angles;
        op->n_bins = d->n_bins;
        op->span = d->angle_span;
        op->M = (int64_t)d->n_angles * d->n_bins;
        st = radon_setup(op);
    } else if (d->kind == NYS_OP_FANBEAM) {
        const double half_diag = 0.5 * std::sqrt((double)d->n1 * d->n1 + (double)d->n2 * d->n2);
        // the kernels index rays with 32-bit ints and put the angle in grid.y
        if (d->n_angles <= 0 || d->n_angles > 65535 || d->n_bins <= 0 ||
            (int64_t)d->n_angles * d->n_bins >= (int64_t(1) << 31) || !(d->angle_span > 0.0) ||
            !(d->src_dist > half_diag + 2.0) || !(d->det_dist > d->src_dist) || !(d->det_spacing > 0.0)) {
            nys_op_destroy(op);
            return fail(ctx, NYS_EINVAL, "fan-beam geometry needs 0 < n_angles <= 65535, n_bins > 0, fewer than "
                                         "2^31 bins, span > 0, src_dist beyond the image, det_dist > src_dist, "
                                         "det_spacing > 0");
        }
        op->n_angles = d->n_angles;
        op->n_bins = d->n_bins;
        op->span = d->angle_span;
        op->src_dist = d->src_dist;
        op->det_dist = d->det_dist;
        op->det_spacing = d->det_spacing;
        op->M = (int64_t)d->n_angles * d->n_bins;
        st = fanbeam_setup(op);
    } else {
        nys_op_destroy(op);
        return fail(ctx, NYS_EINVAL, "unknown operator kind %d", d->kind);
    }
    if (st) {
        nys_op_destroy(op);
        return st;
    }
    *out = op;
    return NYS_OK;
}

int nys_op_destroy(nys_op* op) {
    if (!op) return NYS_OK;
    if (op->ctx) cudaStreamSynchronize(op->ctx->stream);
    void* bufs[] = {op->taps_fwd, op->taps_adj, op->taps_nrm, op->rtab, op->inter, op->lines};
    for (void* b : bufs)
        if (b) cudaFree(b);
    nys_ctx* ctx = op->ctx;
    delete op;
    ctx_release(ctx);
    return NYS_OK;
}

int nys_op_set_kernel(nys_op* op, const double* kernel, int kh, int kw) {
    if (!op || !kernel) return fail(op ? op->ctx : nullptr, NYS_EINVAL, "null argument");
    if (op->kind != NYS_OP_BLUR && op->kind != NYS_OP_BLUR_DECIM)
        return fail(op->ctx, NYS_EINVAL, "nys_op_set_kernel needs a blur operator");
    if (kh != op->kh || kw != op->kw) return fail(op->ctx, NYS_EINVAL, "kernel shape differs from the op's");
    NYS_CK(op->ctx, cudaStreamSynchronize(op->ctx->stream));
    void* bufs[] = {op->taps_fwd, op->taps_adj, op->taps_nrm, op->inter};
    for (void* b : bufs)
        if (b) cudaFree(b);
    op->taps_fwd = op->taps_adj = op->taps_nrm = op->inter = nullptr;
    op->chunk = 0;
    // graphs that captured the old tap tables must be captured again
    ++op->ctx->scratch_gen;
    op->h.assign(kernel, kernel + (size_t)kh * kw);
    return blur_setup(op);
}

int nys_op_autotune(nys_op* op, int batch, int* choice) {
    if (!op || batch < 1) return fail(op ? op->ctx : nullptr, NYS_EINVAL, "nys_op_autotune: null op or batch < 1");
    nys_ctx* ctx = op->ctx;
    const size_t es = dtype_size(op->dtype);
    void* x = nullptr;
    void* y = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = NYS_OK;
    auto cleanup = [&]() {
        if (x) cudaFree(x);
        if (y) cudaFree(y);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t e = cudaMalloc(&x, (size_t)batch * std::max(op->N, op->M) * es);
    if (e == cudaSuccess) e = cudaMalloc(&y, (size_t)batch * std::max(op->N, op->M) * es);
    if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, (size_t)batch * std::max(op->N, op->M) * es, ctx->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(ctx, e, "nys_op_autotune scratch");
    }
    // stages of (knob, candidates), tuned one after the other on the operator
    // pass they affect
    struct Stage {
        int* knob;
        std::vector<int> cand;
    };
    std::vector<Stage> stages;
    int which = 2;
    int* knob = nullptr;   // the one reported through `choice`
    if (op->kind == NYS_OP_RADON) {
        knob = &op->radon_adj_ak;
        stages.push_back({&op->radon_adj_ak, {4, 8, 16}});
        if (batch >= 4) stages.push_back({&op->radon_adj_ib, {4, 1}});
        which = 1;
    } else if (op->kind == NYS_OP_BLUR && op->dtype != NYS_F64) {
        knob = &op->blur_tile;
        stages.push_back({&op->blur_tile, {32, 64}});
    }
    for (const Stage& sg : stages) {
        if (st) break;
        float best = 1e30f;
        int best_v = *sg.knob;
        for (int v : sg.cand) {
            *sg.knob = v;
            if ((st = op_run(op, which, x, y, batch, op->dtype, op->dtype))) break;   // warm-up
            cudaEventRecord(e0, ctx->stream);
            for (int r = 0; r < 3 && !st; ++r) st = op_run(op, which, x, y, batch, op->dtype, op->dtype);
            cudaEventRecord(e1, ctx->stream);
            if (st) break;
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
                st = cuda_fail(ctx, e, "nys_op_autotune timing");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_v = v;
            }
        }
        *sg.knob = best_v;
    }
    cudaStreamSynchronize(ctx->stream);
    cleanup();
    if (choice) *choice = knob ? *knob : 0;
    return st;
}

int nys_op_sizes(const nys_op* op, int64_t* N, int64_t* M) {
    if (!op) return fail(nullptr, NYS_EINVAL, "null op");
    if (N) *N = op->N;
    if (M) *M = op->M;
    return NYS_OK;
}

static int check_io(nys_op* op, const void* a, const void* b, int batch) {
    if (!op) return fail(nullptr, NYS_EINVAL, "null op");
    if (!a || !b) return fail(op->ctx, NYS_EINVAL, "null data pointer");
    if (batch < 0) return fail(op->ctx, NYS_EINVAL, "negative batch");
    return NYS_OK;
}

int op_apply(nys_op* op, const void* x, void* y, int batch) {
    if (int st = check_io(op, x, y, batch)) return st;
    if (batch == 0) return NYS_OK;
    return op_run(op, 0, x, y, batch, op->dtype, op->dtype);
}

int op_adjoint(nys_op* op, const void* y, void* x, int batch) {
    if (int st = check_io(op, y, x, batch)) return st;
    if (batch == 0) return NYS_OK;
    return op_run(op, 1, y, x, batch, op->dtype, op->dtype);
}

int op_normal(nys_op* op, const void* x, void* y, int batch) {
    if (int st = check_io(op, x, y, batch)) return st;
    if (batch == 0) return NYS_OK;
    return op_run(op, 2, x, y, batch, op->dtype, op->dtype);
}

int op_haar(nys_op* op, const void* in, void* out, int batch, int inverse) {
    if (int st = check_io(op, in, out, batch)) return st;
    if (op->haar_levels <= 0) return fail(op->ctx, NYS_EINVAL, "operator was created without haar_levels");
    if (batch == 0) return NYS_OK;
    return haar_run(op, in, out, batch, inverse, op->dtype, op->dtype);
}

int nys_gram(nys_ctx* ctx, int dtype, const void* A, int p, const void* B, int q, int64_t N, double* C, int path) {
    if (!ctx || !A || !B || !C) return fail(ctx, NYS_EINVAL, "nys_gram: null argument");
    if (dtype != NYS_F32 && dtype != NYS_F64 && dtype != NYS_BF16) return fail(ctx, NYS_EINVAL, "nys_gram: dtype");
    if (path < 0 || path > 2) return fail(ctx, NYS_EINVAL, "nys_gram: path");
    if (int st = gram_AtB_path(ctx, dtype, A, p, B, q, N, C, q, path)) return st;
    return check_tc_timeout(ctx);
}

int nys_tall_gemm(nys_ctx* ctx, int in_dtype, const void* A, const void* A2, double alpha, int64_t N, int k,
                  const double* W, int q, int out_dtype, void* out, int path) {
    if (!ctx || !A || !W || !out) return fail(ctx, NYS_EINVAL, "nys_tall_gemm: null argument");
    if (N <= 0 || k <= 0 || q <= 0 || path < 0 || path > 2) return fail(ctx, NYS_EINVAL, "nys_tall_gemm: sizes");
    int st;
    double* a_dev = (double*)scratch(ctx, SLOT_TCERR + 1, 64, &st);
    if (st) return st;
    NYS_CK(ctx, cudaMemcpyAsync(a_dev, &alpha, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if ((st = gemm_tall_path(ctx, in_dtype, A, A2, a_dev, N, k, W, q, out_dtype, out, path))) return st;
    return check_tc_timeout(ctx);
}

int nys_rel_err(nys_ctx* ctx, int dtype, int64_t n, const void* a, const void* b, double* out) {
    if (!ctx || !a || !out) return fail(ctx, NYS_EINVAL, "nys_rel_err: null argument");
    if (dtype != NYS_F32 && dtype != NYS_F64) return fail(ctx, NYS_EINVAL, "nys_rel_err: dtype");
    int st;
    double* dev = nullptr;
    if ((st = norm2_diff(ctx, dtype, n, a, b, &dev))) return st;
    double h[2];
    NYS_CK(ctx, cudaMemcpyAsync(h, dev, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    NYS_CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (b == nullptr) {
        *out = std::sqrt(h[0]);
    } else {
        if (!(h[1] > 0.0)) return fail(ctx, NYS_EINVAL, "nys_rel_err: reference has zero norm");
        *out = std::sqrt(h[0] / h[1]);
    }
    return NYS_OK;
}

}  // extern "C"
