// Many differentiated unrolled solves as one CUDA graph.
//
// Each item is an nys_unroll handle bound to its own context (own stream and
// scratch), with its data, output, cotangent and gradient buffers fixed at
// creation.  nys_batch_create runs every item's forward and reverse pass once
// outside capture (which sizes every scratch region and sets every kernel
// attribute), then captures two graphs on the batch context's stream: the
// stream forks to every item's stream (an event), each item records its
// launches there, and the item streams join back.  The items become parallel
// branches of one graph, so nys_batch_forward / nys_batch_backward are one
// cudaGraphLaunch each, whatever the number, sizes and operators of the
// items.
#include "internal.cuh"

#include <vector>

struct nys_batch {
    nys_ctx* ctx = nullptr;
    std::vector<nys_unroll*> items;
    std::vector<nys_ctx*> item_ctx;
    std::vector<const void*> ys;
    std::vector<void*> xs;
    std::vector<const void*> xbars;
    std::vector<double*> grads;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t g_fwd = nullptr, g_bwd = nullptr;
    bool fwd_done = false;
    uint64_t gen = 0;   // sum of the item contexts' scratch generations at capture
};

namespace nys {
namespace {

int run_items(nys_batch* B, bool backward, bool captured) {
    cudaStream_t main = B->ctx->stream;
    int st = NYS_OK;
    if (captured) NYS_CK(B->ctx, cudaEventRecord(B->fork, main));
    for (size_t i = 0; i < B->items.size() && !st; ++i) {
        cudaStream_t si = B->item_ctx[i]->stream;
        if (captured) {
            cudaError_t e = cudaStreamWaitEvent(si, B->fork, 0);
            if (e != cudaSuccess) return cuda_fail(B->ctx, e, "batch fork");
        }
        st = backward ? nys_unroll_backward(B->items[i], B->xbars[i], B->grads[i])
                      : nys_unroll_forward(B->items[i], B->ys[i], B->xs[i]);
        if (st) {
            fail(B->ctx, st, "batch item %zu: %s", i, nys_last_error(B->item_ctx[i]));
            break;
        }
        if (captured) {
            cudaError_t e = cudaEventRecord(B->joins[i], si);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(main, B->joins[i], 0);
            if (e != cudaSuccess) return cuda_fail(B->ctx, e, "batch join");
        }
    }
    return st;
}

int capture(nys_batch* B, bool backward, cudaGraphExec_t* out) {
    cudaStream_t main = B->ctx->stream;
    NYS_CK(B->ctx, cudaStreamBeginCapture(main, cudaStreamCaptureModeRelaxed));
    const int st = run_items(B, backward, true);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(main, &g);
    if (st || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st ? st : cuda_fail(B->ctx, e, "batch capture");
    }
    const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return cuda_fail(B->ctx, ei, "batch graph instantiate");
    return NYS_OK;
}

// the graphs hold the addresses of the item contexts' scratch regions
uint64_t scratch_gens(const nys_batch* B) {
    uint64_t g = B->ctx->scratch_gen;
    for (nys_ctx* c : B->item_ctx) g += c->scratch_gen;
    return g;
}

// capture both graphs again if a scratch region they use was reallocated
int refresh(nys_batch* B) {
    if (B->gen == scratch_gens(B)) return NYS_OK;
    for (nys_ctx* c : B->item_ctx) NYS_CK(B->ctx, cudaStreamSynchronize(c->stream));
    NYS_CK(B->ctx, cudaStreamSynchronize(B->ctx->stream));
    cudaGraphExec_t f = nullptr, b = nullptr;
    int st = capture(B, false, &f);
    if (!st) st = capture(B, true, &b);
    if (st) {
        if (f) cudaGraphExecDestroy(f);
        return st;
    }
    cudaGraphExecDestroy(B->g_fwd);
    cudaGraphExecDestroy(B->g_bwd);
    B->g_fwd = f;
    B->g_bwd = b;
    B->gen = scratch_gens(B);
    return NYS_OK;
}

}  // namespace
}  // namespace nys

using namespace nys;

extern "C" {

int nys_batch_create(nys_ctx* ctx, int n, nys_unroll* const* items, nys_ctx* const* item_ctx,
                     const void* const* ys, void* const* xs, const void* const* xbars, double* const* grads,
                     nys_batch** out) {
    if (!ctx || n < 1 || !items || !item_ctx || !ys || !xs || !xbars || !grads || !out)
        return fail(ctx, NYS_EINVAL, "nys_batch_create: null argument or n < 1");
    *out = nullptr;
    if (!ctx->stream) return fail(ctx, NYS_EINVAL, "nys_batch_create: the batch context needs its own stream");
    for (int i = 0; i < n; ++i) {
        if (!items[i] || !item_ctx[i] || !ys[i] || !xs[i] || !xbars[i] || !grads[i])
            return fail(ctx, NYS_EINVAL, "nys_batch_create: item %d has a null pointer", i);
        if (!item_ctx[i]->stream || item_ctx[i]->stream == ctx->stream)
            return fail(ctx, NYS_EINVAL, "nys_batch_create: item %d needs a stream of its own", i);
        nys_ctx *uc = nullptr, *oc = nullptr;
        unroll_contexts(items[i], &uc, &oc);
        if (uc != item_ctx[i] || oc != item_ctx[i])
            return fail(ctx, NYS_EINVAL, "nys_batch_create: item %d and its operator must use item_ctx[%d]", i, i);
    }
    nys_batch* B = new nys_batch();
    B->ctx = ctx;
    ctx_retain(ctx);
    B->items.assign(items, items + n);
    B->item_ctx.assign(item_ctx, item_ctx + n);
    B->ys.assign(ys, ys + n);
    B->xs.assign(xs, xs + n);
    B->xbars.assign(xbars, xbars + n);
    B->grads.assign(grads, grads + n);
    B->joins.resize(n, nullptr);
    cudaError_t e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&B->joins[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        nys_batch_destroy(B);
        return cuda_fail(ctx, e, "nys_batch_create events");
    }
    // one uncaptured pass of every item: sizes all scratch, sets attributes
    int st = run_items(B, false, false);
    if (!st) st = run_items(B, true, false);
    for (int i = 0; i < n && !st; ++i)
        if (cudaStreamSynchronize(B->item_ctx[i]->stream) != cudaSuccess) st = cuda_fail(ctx, cudaGetLastError(), "batch warm-up");
    if (!st) st = capture(B, false, &B->g_fwd);
    if (!st) st = capture(B, true, &B->g_bwd);
    B->gen = scratch_gens(B);
    if (st) {
        nys_batch_destroy(B);
        return st;
    }
    *out = B;
    return NYS_OK;
}

int nys_batch_forward(nys_batch* B) {
    if (!B) return fail(nullptr, NYS_EINVAL, "null batch");
    if (int st = refresh(B)) return st;
    NYS_CK(B->ctx, cudaGraphLaunch(B->g_fwd, B->ctx->stream));
    B->fwd_done = true;
    return NYS_OK;
}

int nys_batch_backward(nys_batch* B) {
    if (!B) return fail(nullptr, NYS_EINVAL, "null batch");
    if (!B->fwd_done) return fail(B->ctx, NYS_EINVAL, "nys_batch_backward before nys_batch_forward");
    if (int st = refresh(B)) return st;
    NYS_CK(B->ctx, cudaGraphLaunch(B->g_bwd, B->ctx->stream));
    return NYS_OK;
}

int nys_batch_destroy(nys_batch* B) {
    if (!B) return NYS_OK;
    if (B->ctx) cudaStreamSynchronize(B->ctx->stream);
    if (B->g_fwd) cudaGraphExecDestroy(B->g_fwd);
    if (B->g_bwd) cudaGraphExecDestroy(B->g_bwd);
    if (B->fork) cudaEventDestroy(B->fork);
    for (cudaEvent_t ev : B->joins)
        if (ev) cudaEventDestroy(ev);
    nys_ctx* ctx = B->ctx;
    delete B;
    ctx_release(ctx);
    return NYS_OK;
}

}  // extern "C"
