// Internal declarations shared by the CUDA translation units of libnys.
// Nothing here is part of the C ABI (include/nys.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

#include "../../include/nys.h"

namespace nys {

// ----------------------------------------------------------- numerics ----
__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ double ldf(const double* p) { return *p; }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void stf(float* p, float v) { *p = v; }
__device__ __forceinline__ void stf(double* p, double v) { *p = v; }
__device__ __forceinline__ void stf(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void stf(float* p, double v) { *p = (float)v; }
__device__ __forceinline__ void stf(__nv_bfloat16* p, double v) { *p = __float2bfloat16_rn((float)v); }

// compute type: double for double storage, float otherwise
template <class T> struct Comp { using type = float; };
template <> struct Comp<double> { using type = double; };

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; `sh` needs blockDim.x/32 entries.  Result valid in
// every thread.  Must be called by all threads of the block.
template <class T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T r = (threadIdx.x < (unsigned)nw) ? sh[threadIdx.x] : T(0);
    if (wid == 0) r = warp_sum(r);
    if (threadIdx.x == 0) sh[0] = r;
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}

__host__ __device__ __forceinline__ int pmod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

inline size_t dtype_size(int dt) { return dt == NYS_F64 ? 8 : (dt == NYS_BF16 ? 2 : 4); }

}  // namespace nys

// ----------------------------------------------------------- handles -----
struct nys_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 152;
    int64_t l2_bytes = 0;   // device L2 size (cudaDevAttrL2CacheSize)
    int64_t launches = 0;   // kernels launched through this context
    cudaStreamAttrValue l2_window = {};   // access-policy window set by nys_l2_persist
    bool l2_window_set = false;
    std::string err;
    unsigned* counters = nullptr;   // device, COUNTER_WORDS words: completion counters (vec.cuh), dual-stop flags
    // exact early stop of the anisotropic-TV dual iteration (DualStop below),
    // on unless nys_set_dual_stop turned it off
    bool dual_stop = true;
    // the context is freed when its owner (nys_destroy) and every object
    // created on it (operators, solvers, unrolled solves, batches) are gone,
    // in whatever order they are destroyed
    int refs = 1;
    // independent growable scratch regions (see nys::scratch)
    void* slot_ptr[12] = {nullptr};
    size_t slot_bytes[12] = {0};
    // incremented whenever a scratch region is reallocated: a CUDA graph that
    // captured the old address must be captured again before it is replayed
    uint64_t scratch_gen = 0;
};

struct nys_op {
    nys_ctx* ctx = nullptr;
    int kind = 0, dtype = 0, n1 = 0, n2 = 0;
    int64_t N = 0, M = 0;
    int haar_levels = 0;
    int wavelet = 0;                  // NYS_WAVELET_HAAR or NYS_WAVELET_DB4
    // blur
    int kh = 0, kw = 0, decim = 1;
    std::vector<double> h;            // kh*kw
    bool separable = false;
    // device tap tables (dtype of the op): see blur.cu
    void* taps_fwd = nullptr;         // H   (2-D kernel or [col taps | row taps])
    void* taps_adj = nullptr;         // H^T
    void* taps_nrm = nullptr;         // H^T H (separable only)
    int Lc_f = 0, Lr_f = 0, cc_f = 0, cr_f = 0;   // separable forward lengths/centres
    int Lc_n = 0, Lr_n = 0, cc_n = 0, cr_n = 0;   // separable normal
    // radon
    int n_angles = 0, n_bins = 0;
    double span = 0.0;
    void* rtab = nullptr;             // per-angle tables, see radon.cu
    void* lines = nullptr;            // radon: `chunk` images as line-major copies (row-major and transposed)
    double src_dist = 0.0, det_dist = 0.0, det_spacing = 1.0;   // fan beam
    int radon_adj_ak = 16;            // radon adjoint: angles per round, 4, 8 or 16 (nys_op_autotune)
    int radon_adj_ib = 4;             // radon adjoint: images per CTA for batches of 4 or more, 1 or 4
    int blur_tile = 64;               // blur: output tile side, 32 or 64 (float32; chosen by nys_op_autotune)
    // intermediate buffer for two-pass normals (M per image, `chunk` images)
    void* inter = nullptr;
    int chunk = 0;
};

namespace nys {

// reference counting of a context by the objects created on it
void ctx_retain(nys_ctx* ctx);
void ctx_release(nys_ctx* ctx);
// record an error on ctx (and globally) and return `code`
int fail(nys_ctx* ctx, int code, const char* fmt, ...);
int cuda_fail(nys_ctx* ctx, cudaError_t e, const char* what);
// Number of leading active columns of U (N values of es bytes each) whose
// loads carry the L2 evict_last priority, so that they stay in L2 between the
// many P^{-1} applications of a solve while the other columns stream past
// with evict_first: all le columns when U fits in the L2 budget (a fraction
// of the L2 size, NYS_L2_KEEP, default 0.5), else as many as fit.
int l2_keep_cols(const nys_ctx* ctx, int64_t N, size_t es, int le);
// Opt `func` in to `bytes` of dynamic shared memory on ctx's device (the
// current device), once per kernel and device; NYS_OK or NYS_ECUDA.
int smem_optin(nys_ctx* ctx, const void* func, size_t bytes);

// Scratch regions: each slot is an independent buffer that grows on demand.
enum Slot {
    SLOT_PRECOND = 0,   // partial sums of U^T z
    SLOT_PROX = 1,      // dual variables of prox_tv / prox_hs
    SLOT_FACTOR = 2,    // ell x ell work in nys_factor
    SLOT_SSN = 3,       // semi-smooth Newton state
    SLOT_MISC = 4,      // reductions, converted GEMM operands
    SLOT_OPTMP = 5,     // Haar ping-pong buffers
    SLOT_SKETCH = 6,    // W^T Omega and A^T A W^T Omega in nys_sketch
    SLOT_GRAM = 7,      // split-K partial tiles of gram_AtB
    SLOT_SOLVER = 8,    // solver temporaries
    SLOT_EIG = 9,       // Jacobi rotation log
    SLOT_TCERR = 10,    // time-out flag of the tensor-core kernels
    SLOT_COUNT = 11
};
void* scratch(nys_ctx* ctx, int slot, size_t bytes, int* status);
// elements of SLOT_PROX the dual prox needs for G dual components over N
// pixels: two (R, Q) buffers and two images
inline size_t prox_work_elems(int G, int64_t N) { return (size_t)(4 * G + 2) * (size_t)N; }

#define NYS_CK(ctx, call)                                              \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return nys::cuda_fail((ctx), e_, #call); \
    } while (0)

// ------------------------------------ programmatic dependent launch ----
// The kernels of the iteration are short (a few µs at 512²) and run back to
// back in one stream or graph, so the gap between two of them is a large part
// of an iteration.  A kernel launched through launch_pdl() may be scheduled
// while its predecessor in the stream is still running; it must then begin
// with pdl_enter(), whose griddepcontrol.wait returns only once every grid
// it depends on has completed and its writes are visible (a no-op for a
// normal launch), before it touches memory.  The trigger after it lets the
// next kernel be scheduled in turn.  Because every such kernel waits before
// any access, completion stays transitive along the stream.
// The attribute is set on eager launches only: replayed from a CUDA graph the
// same kernels ran about 4% slower with it on a GB300 (the graph already
// removes the launch gaps).  NYS_PDL in the environment: 0 = never, 2 = also
// while a stream is being captured, otherwise eager launches only.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

int pdl_mode();   // api.cu: 0, 1 or 2 as above

// Exact early stop of the dual APG of the mixed-norm proxes (TV, isotropic
// TV, HS_1, HS_2, HS_inf).  A dual step maps (R, Q) to (R', Q') by a fixed
// deterministic function of (R, Q) and of beta, and beta only multiplies
// Q' - Q.  If a step leaves every component unchanged (Q' = R = Q), every
// later step reproduces it exactly, so once a step j >= 1 has changed
// nothing, steps j + 1 ... may be skipped: the buffers (ping-pong or updated
// in place) already hold the fixed point, and the result is bit-identical to
// running them.  (In the fused anisotropic-TV step, step 0's input g comes
// from a differently ordered L^T, so step 0 does not count.)
// Three flags in ctx->counters: step k sets flag k % 3 when any component
// changed and clears flag (k + 1) % 3 for step k + 1; step k >= 2 is skipped
// when flag (k - 1) % 3 is clear.  A skipped last step still writes Q (and,
// without a preconditioner, the output x) out.  Each flag is spread over
// DUAL_STOP_SLOTS words (block b sets word b % DUAL_STOP_SLOTS): a thousand
// blocks storing to one word serialise for tens of microseconds.
constexpr int COUNTER_DUAL_SKIPPED = 8;     // dual steps skipped (wraps)
constexpr int DUAL_STOP_SLOTS = 128;
constexpr int COUNTER_DUAL_STOP = 512;      // 3 x DUAL_STOP_SLOTS flag words
constexpr int COUNTER_WORDS = COUNTER_DUAL_STOP + 3 * DUAL_STOP_SLOTS;   // ctx->counters size
struct DualStop {
    unsigned* flags = nullptr;   // nullptr: this launch never skips
    int k = 0;                   // the dual step of this launch
    // the x pass of a skipped last step: where the fixed point's x already is
    // (the pass copies it to its output instead of streaming U again)
    const void* copy = nullptr;
};
// Whether this launch's step is skipped, the same answer in every thread of
// the block: every thread calls it (a block barrier when armed), blockDim.x
// >= DUAL_STOP_SLOTS
__device__ __forceinline__ bool dual_skip(const DualStop& s) {
    if (!s.flags || s.k < 2) return false;   // a kernel parameter: the same in every thread
    int set = 0;
    if (threadIdx.x < DUAL_STOP_SLOTS)
        set = *(volatile const unsigned*)(s.flags + ((s.k + 2) % 3) * DUAL_STOP_SLOTS + threadIdx.x) != 0u;
    return !__syncthreads_or(set);
}
// the step's own bookkeeping, by block 0: clear the next step's flag and
// count a skip
__device__ __forceinline__ void dual_stop_enter(const DualStop& s, bool skip) {
    if (s.flags && blockIdx.x == 0 && blockIdx.y == 0) {
        if (threadIdx.x < DUAL_STOP_SLOTS) s.flags[((s.k + 1) % 3) * DUAL_STOP_SLOTS + threadIdx.x] = 0u;
        if (skip && threadIdx.x == 0) atomicAdd(s.flags + (COUNTER_DUAL_SKIPPED - COUNTER_DUAL_STOP), 1u);
    }
}
// a step that computed: set its flag when any thread of the block saw a change
// (every thread of the block calls this; a block barrier)
__device__ __forceinline__ void dual_stop_report(const DualStop& s, bool changed) {
    if (!s.flags) {
        __syncthreads();
        return;
    }
    const int any = __syncthreads_or(changed ? 1 : 0);
    if (s.flags && any && threadIdx.x == 0) s.flags[(s.k % 3) * DUAL_STOP_SLOTS + blockIdx.x % DUAL_STOP_SLOTS] = 1u;
}

inline bool pdl_enabled(cudaStream_t stream) {
    const int m = pdl_mode();
    if (m == 0) return false;
    if (m == 2) return true;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled(stream) ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

#define NYS_LAUNCH_CK(ctx)                                             \
    do {                                                               \
        (ctx)->launches += 1;                                          \
        cudaError_t e_ = cudaGetLastError();                           \
        if (e_ != cudaSuccess) return nys::cuda_fail((ctx), e_, "kernel launch"); \
    } while (0)

// ------------------------------------------------ internal launch API ----
// operators (blur.cu, radon.cu, haar.cu)
int blur_setup(nys_op* op);
int blur_run(nys_op* op, int which /*0 fwd,1 adj,2 normal*/, const void* x, void* y, int batch,
             int in_dtype, int out_dtype);
int decim_run(nys_op* op, int which, const void* x, void* y, int batch, int in_dtype, int out_dtype);
int radon_setup(nys_op* op);
int radon_run(nys_op* op, int which, const void* x, void* y, int batch, int in_dtype, int out_dtype);
int fanbeam_setup(nys_op* op);
int fanbeam_run(nys_op* op, int which, const void* x, void* y, int batch, int in_dtype, int out_dtype);
int haar_run(nys_op* op, const void* in, void* out, int batch, int inverse, int in_dtype, int out_dtype);
// generic: which = 0 A, 1 A^T, 2 A^T A ; dtypes may differ from op dtype (bf16 io)
int op_run(nys_op* op, int which, const void* x, void* y, int batch, int in_dtype, int out_dtype);

// dense helpers (dense.cu)
// C[p x q] (double) = A^T B, A: N x p, B: N x q (column j at offset j*N)
int gram_AtB(nys_ctx* ctx, int dtype, const void* A, int p, const void* B, int q, int64_t N,
             double* C, int ldc);
// path: 0 = tensor cores when the shape allows, 1 = CUDA cores, 2 = tensor cores or NYS_EINVAL
int gram_AtB_path(nys_ctx* ctx, int dtype, const void* A, int p, const void* B, int q, int64_t N, double* C, int ldc,
                  int path);
// tcgen05 Gram for bf16 operands (gram_tc.cu); NYS_EINVAL when unsupported
int gram_AtB_tc(nys_ctx* ctx, const void* A, int p, const void* B, int q, int64_t N, double* C, int ldc);
// one product srcs[a]^T srcs[b] into C (float64, ld = ldc) of a multi-product launch
struct GramJob {
    int a, b;
    double* C;
    int ldc;
};
// up to four Gram products of up to two bf16 operands (cols[s] columns of N
// pixels, at most 1024) in one tensor-core launch (gram_tc.cu); NYS_EINVAL
// when unsupported
int gram_tc_jobs(nys_ctx* ctx, const void* const* srcs, const int* cols, int nsrc, int64_t N, int njobs,
                 const GramJob* jobs);
void gram_reduce_f32(nys_ctx* ctx, const float* part, int splits, int p, int q, double* C, int ldc, int blocks);
// tcgen05 U = (Y + v Omega) W for bf16 Y, Omega, ell <= 1024 (gram_tc.cu); NYS_EINVAL when unsupported
int gemm_tall_tc(nys_ctx* ctx, const void* Y, const void* Om, const double* v_dev, int64_t N, int ell,
                 const double* W, int out_dt, void* out);
// path: 0 = tensor cores when possible, 1 = CUDA cores, 2 = tensor cores or NYS_EINVAL
int gemm_tall_path(nys_ctx* ctx, int in_dt, const void* A, const void* A2, const double* alpha_dev, int64_t N,
                   int k, const double* W, int q, int out_dt, void* out, int path);
// raise NYS_ETIMEOUT if a tensor-core kernel recorded a time-out (synchronises)
int check_tc_timeout(nys_ctx* ctx);
// out (N x q, dtype out_dt) = (A + alpha*A2) W, A/A2: N x k of in_dt, W: k x q double (row-major k x q)
int gemm_tall(nys_ctx* ctx, int in_dt, const void* A, const void* A2, const double* alpha_dev, int64_t N,
              int k, const double* W, int q, int out_dt, void* out);

// eigenvectors V (float32, row-major, ld = ldv) of the symmetric ell x ell
// float64 G by one-sided Jacobi on a thread-block cluster
// (jacobi_cluster.cu), Rsave = ell * ell floats of workspace; NYS_EINVAL
// (nothing launched) when not applicable; *status (device) = 1 if the
// float32 Cholesky of G fails
int jacobi_cluster(nys_ctx* ctx, const double* G, int ell, int max_sweeps, float* V, int ldv, float* Rsave,
                   int* sweeps, int* status);

// float64 Cholesky L (n x n, lower, row-major) on a 16-CTA cluster
// (chol_cluster.cu): mode 0 of src (ld), status in info[slot]; mode 1 of
// sym(Omega^T Y) + v Omega^T Omega from the Gram src = G2 with the shift and
// its retries in info[0..2].  NYS_EINVAL (nothing launched) when n is outside
// [48, 512] or the cluster cannot be placed.
int chol_cluster(nys_ctx* ctx, const double* src, int ld, int n, int mode, double eps, int max_retries, double* L,
                 double* info, int slot);

// Omega for Algorithm 1 step 1: total i.i.d. N(0,1) entries (factor.cu)
int omega_fill(nys_ctx* ctx, int store_dt, void* Omega, int64_t total, uint64_t seed, int64_t first = 0);

// reductions (reduce.cu)
int norm2_diff(nys_ctx* ctx, int dtype, int64_t n, const void* a, const void* b, double** out_dev);

}  // namespace nys

// precond internal state (precond.cu)
struct nys_precond_priv {
    double* K = nullptr;      // ell x ell, U^T U
    double* d = nullptr;      // ell weights
    double* M64 = nullptr;    // ell x ell, inverse-apply matrix
    float* M32 = nullptr;
    float* d32 = nullptr;
    double* sqrtd = nullptr;  // ell, sqrt(d) (Ubar scaling)
    int ell = 0;
    // d is non-increasing (S_hat is sorted), so only the columns j < ell_eff
    // with d_j > 0 enter P and P^{-1}; the rows and columns of M beyond it are 0
    int ell_eff = 0;
};

namespace nys {
// P^{-1} or P applied to z (dtype f32/f64); out may alias z.  If `lt_src` is
// not null the input is computed on the fly (used by the fused prox kernels).
int precond_run(nys_ctx* ctx, const nys_precond* pc, int inverse, int dtype, const void* z,
                void* out, int batch);
// the contexts an unrolled-solve handle launches on (unroll.cu)
void unroll_contexts(const nys_unroll* U, nys_ctx** ctx, nys_ctx** op_ctx);
// dual APG prox with the fused two-launch (TV) or three-launch (HS) step
// (prox_fused.cu); returns
// NYS_EINVAL without launching anything when the layout does not allow it
int prox_dual_fused(nys_ctx* ctx, const nys_precond* pc, int reg, double lb, int n_inner, int dtype, int n1, int n2,
                    const void* s, void* out, void* Q);
}  // namespace nys
