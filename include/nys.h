/*
 * nys.h -- C ABI of the GB300 randomized-Nystrom-preconditioned reconstruction
 * library (arxiv 2411.08178, "randomized Nystrom preconditioners for
 * variational image reconstruction").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Pointers.   Arguments named x, y, z, s, out, Omega, Y, U, Q, S_hat, gamma are
 *             DEVICE pointers owned by the caller; the library never frees
 *             them.  Descriptor structs and scalars are host memory.
 * Layout.     An image is n1 x n2, row-major (pixel (i, j) = row i, column j at
 *             offset i*n2 + j).  A batch of B images is B images back to back.
 *             An N x ell matrix (Omega, Y, U) is stored as ell images back to
 *             back, since every probe column is itself an image (Sec. III-C):
 *             column j starts at offset j*N.
 * Types.      dtype NYS_F64 or NYS_F32 for images; the sketch may also use
 *             NYS_BF16 storage for Omega, Y and U (FP32 accumulation).
 * Streams.    Every call is asynchronous on the context's CUDA stream unless
 *             it says otherwise; host-visible results are noted per call.
 * Memory.     op_apply / op_adjoint / op_normal, precond_apply, prox_* and
 *             pgd_step never allocate: their scratch comes from the context
 *             workspace, which nys_reserve() sizes ahead of time (calls made
 *             before a reserve may grow it once).  Growing a region frees its
 *             old buffer: the CUDA graphs that solvers and batches capture
 *             are captured again before their next replay, but a graph the
 *             caller captures itself must be captured again by the caller
 *             (or the workspace reserved before capturing).
 * Errors.     Every function returns NYS_OK (0) or one of the codes below and
 *             records a message readable with nys_last_error().  No C++
 *             exception crosses this boundary.  A NULL handle or required
 *             pointer gives NYS_EINVAL before any device work; the
 *             *_destroy / *_release functions accept NULL and do nothing.
 */
#ifndef NYS_H
#define NYS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes -- */
enum {
    NYS_OK = 0,
    NYS_EINVAL = 1,        /* bad shape, dtype, null pointer or argument      */
    NYS_ENOMEM = 2,        /* device allocation failed                        */
    NYS_ECUDA = 3,         /* a CUDA runtime call failed                      */
    NYS_ENOTSPD = 4,       /* Cholesky of the shifted core failed 8 retries   */
    NYS_EDEGENERATE = 5,   /* s_K + mu <= 0 in the preconditioner             */
    NYS_ENONFINITE = 6,    /* NaN/Inf produced                                */
    NYS_ETIMEOUT = 7,      /* a bounded device wait ran out                   */
    NYS_ENOCONV = 8        /* iteration cap hit (warning: output still valid) */
};

enum { NYS_F32 = 0, NYS_F64 = 1, NYS_BF16 = 2 };
enum { NYS_OP_BLUR = 0, NYS_OP_BLUR_DECIM = 1, NYS_OP_RADON = 2, NYS_OP_FANBEAM = 3 };
enum { NYS_PHI_ATA = 0, NYS_PHI_W_ATA_WT = 1 };
/* regularisers ||L x||_{1,phi} (Eq. lpl1qMixedNorm, Appendix A): Haar l1;
 * first differences with phi = 1 (anisotropic TV) or phi = 2 (isotropic TV);
 * the 2x2 Hessian with the Schatten-1, -2 or -inf norm (HS_1, HS_2, HS_inf) */
enum { NYS_WAVELET_HAAR = 0, NYS_WAVELET_DB4 = 1 };
enum { NYS_REG_WAVELET = 0, NYS_REG_TV = 1, NYS_REG_HS = 2, NYS_REG_ISOTV = 3, NYS_REG_HS2 = 4, NYS_REG_HSINF = 5 };
enum { NYS_FIT_L2 = 0, NYS_FIT_HUBER = 1 };

typedef struct nys_ctx nys_ctx;
typedef struct nys_op nys_op;
typedef struct nys_solver nys_solver;

/* ------------------------------------------------------------- context -- */
/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  *ctx is set on success. */
int nys_create(nys_ctx** ctx, int device, void* cuda_stream);
int nys_destroy(nys_ctx* ctx);
/* Replace the stream used by later calls on this context. */
int nys_set_stream(nys_ctx* ctx, void* cuda_stream);
/* Block the host until all work issued on the context's stream is done. */
int nys_sync(nys_ctx* ctx);
/* Message of the last failing call on this context ("" if none).  Valid until
 * the next call on the same context.  NULL ctx gives the global message. */
const char* nys_last_error(const nys_ctx* ctx);
/* Make sure the context workspace holds at least `bytes` bytes. */
int nys_reserve(nys_ctx* ctx, size_t bytes);
/* Library version string. */
const char* nys_version(void);
/* Keep [ptr, ptr + bytes) resident in L2 for kernels issued on the context's
 * stream (and in graphs the solvers capture afterwards): reserves the
 * device's largest persisting-L2 carve-out for this CUDA context and sets the
 * stream's access-policy window (persisting hits, streaming misses).
 * hit_ratio scales the fraction of the window marked persisting.  ptr = NULL
 * clears the window.  The setting belongs to this process's CUDA context and
 * ends with it.  Needs a non-default stream. */
int nys_l2_persist(nys_ctx* ctx, const void* ptr, size_t bytes, double hit_ratio);
/* Number of kernels launched through this context since it was created. */
int nys_launch_count(const nys_ctx* ctx, int64_t* count);
/* Exact early stop of the dual APG of the mixed-norm proxes (prox_tv,
 * prox_hs, prox_mixed; Sec. III-B, the dual problem solved by APG), on by
 * default: once a dual step j >= 1
 * leaves every component of the dual iterate and of its extrapolation
 * unchanged, every later step would reproduce it (a step is a deterministic
 * function of that pair), so the remaining steps of the call are skipped on
 * the device and the result is bit-identical to running all n_inner steps.
 * on = 0 runs every step.  Takes effect for prox calls issued, and solver
 * iterations captured, after the call; NYS_EINVAL for a null context. */
int nys_set_dual_stop(nys_ctx* ctx, int on);
/* Dual steps skipped by the early stop on this context so far (a 32-bit
 * device counter, wraps); synchronises the context's stream. */
int nys_dual_steps_skipped(nys_ctx* ctx, int64_t* count);

/* ------------------------------------------------------------ operators -- */
/* Forward models of Sec. IV: periodic blur (IV-A), blur + decimation
 * (IV-A, super-resolution) and the parallel-beam ray transform (IV-C),
 * discretised with Joseph's method: ray (theta_k, t_m) with
 * theta_k = k * angle_span / n_angles, detector offset t_m = m - (n_bins-1)/2
 * pixels, pixel (i, j) at x = j - (n2-1)/2, y = i - (n1-1)/2; one sample per
 * row (|cos| + 1e-9 >= |sin|, weight 1/|cos|) or per column (weight 1/|sin|)
 * with linear interpolation, zero outside the image.
 * Fan beam (NYS_OP_FANBEAM, the experiments' second CT geometry): a point
 * source on a circle of radius src_dist about the image centre and a flat
 * detector at det_dist from it; at angle theta_k = k * angle_span / n_angles
 * the source sits at R (cos, sin) and bin m at offset (m - (n_bins-1)/2)
 * det_spacing along (-sin, cos) on the detector; each ray is sampled by
 * Joseph's method along rows (|d_y| >= |d_x|) or columns, weight |d| / |major
 * component|.  src_dist must exceed the image half-diagonal by 2 pixels,
 * n_angles <= 65535, and float32 fan-beam operators take images of at most
 * 2048 rows and columns (they evaluate sample positions in float32 split
 * into an integer and a fraction; float64 ones in float64).  Both ray transforms need n_angles * n_bins < 2^31
 * and N = n1 * n2 < 2^31; other sizes return NYS_EINVAL.
 * Blur: (Hx)[i,j] = sum_ab kernel[a*kw+b] x[(i+a-(kh-1)/2) mod n1,
 * (j+b-(kw-1)/2) mod n2]; kh, kw odd.  Decimation keeps pixels (d i, d j).
 * The kernel (host, float64, kh*kw) is copied; the descriptor may be freed
 * after the call.  haar_levels > 0 enables the orthonormal wavelet transform
 * W (Mallat layout, periodic) used by NYS_PHI_W_ATA_WT and the wavelet
 * regulariser (Sec. III-B, invertible L): Haar, or Daubechies' four-tap
 * filter bank (wavelet = NYS_WAVELET_DB4: lo[i] = sum_k h[k] x[(2i+k) mod n],
 * hi with g[k] = (-1)^k h[3-k], columns first); n1, n2 must be divisible by
 * 2^haar_levels. */
typedef struct nys_op_desc {
    int kind;               /* NYS_OP_*                                     */
    int dtype;              /* NYS_F32 or NYS_F64                           */
    int n1, n2;             /* image rows, columns                          */
    const double* kernel;   /* host, kh*kw row-major (blur kinds)           */
    int kh, kw;
    int decim;              /* NYS_OP_BLUR_DECIM factor (n1, n2 divisible)  */
    int n_angles, n_bins;   /* NYS_OP_RADON                                 */
    double angle_span;      /* NYS_OP_RADON, radians (pi = parallel beam)   */
    int haar_levels;        /* 0 = no wavelet                               */
    int wavelet;            /* NYS_WAVELET_HAAR (0) or NYS_WAVELET_DB4      */
    double src_dist;        /* NYS_OP_FANBEAM: source to image centre, R    */
    double det_dist;        /* NYS_OP_FANBEAM: source to detector, D > R    */
    double det_spacing;     /* NYS_OP_FANBEAM: detector bin width           */
} nys_op_desc;

int nys_op_create(nys_ctx* ctx, const nys_op_desc* desc, nys_op** op);
int nys_op_destroy(nys_op* op);
/* Number of pixels N = n1*n2 and measurements M of one image. */
int nys_op_sizes(const nys_op* op, int64_t* N, int64_t* M);
/* Replace the blur kernel (host, float64, kh*kw with the op's kh, kw; copied)
 * of a blur or blur + decimation op.  Synchronises the ctx stream; not
 * capturable.  NYS_EINVAL for other kinds or another kernel shape. */
int nys_op_set_kernel(nys_op* op, const double* kernel, int kh, int kw);

/* Project autotuner: times the operator's launch variants on scratch data
 * of `batch` images (batch >= 1) on the ctx stream and keeps the fastest for
 * this op -- the blur output tile (32 or 64 pixels square, float32 ops) or,
 * for the Radon adjoint, the number of angles per round (4, 8 or 16) and then,
 * for batch >= 4, the images per CTA (4 or 1).  *choice (may be NULL)
 * receives the value kept for the first knob (tile side or angles per round).
 * Allocates and frees scratch and synchronises; not capturable.  Results are
 * the same for every variant up to float summation order. */
int nys_op_autotune(nys_op* op, int batch, int* choice);

/* y[b] = A x[b], b < batch.  x: batch*N, y: batch*M, op dtype. */
int op_apply(nys_op* op, const void* x, void* y, int batch);
/* x[b] = A^T y[b]: the exact transpose of op_apply. */
int op_adjoint(nys_op* op, const void* y, void* x, int batch);
/* y[b] = A^T A x[b] (fused where the operator allows).  x, y: batch*N. */
int op_normal(nys_op* op, const void* x, void* y, int batch);
/* c[b] = W x[b] (inverse = 0) or x[b] = W^T c[b] (inverse = 1). */
int op_haar(nys_op* op, const void* in, void* out, int batch, int inverse);

/* ---------------------------------------------------------- Algorithm 1 -- */
/* Steps 1-2 of Algorithm 1: draw Omega (N x ell, i.i.d. N(0,1)) from the
 * Philox4x32-10 counter generator (element (i, j) -> flat index e = j*N + i,
 * Philox block e/4 with counter (e/4 mod 2^32, e/4 >> 32, 0, 0) and key
 * (seed mod 2^32, seed >> 32), uniforms ((x >> 9) + 0.5) 2^-23, Box-Muller
 * pairs) and write Y = Phi Omega with Phi = A^T A (NYS_PHI_ATA) or
 * W A^T A W^T (NYS_PHI_W_ATA_WT, Sec. III-B).  Omega and Y use `store_dtype`
 * (the op dtype, or NYS_BF16 for an FP32 op: the operator then computes in
 * FP32 and rounds its output). */
int nys_sketch(nys_ctx* ctx, nys_op* op, int phi_kind, int ell, uint64_t seed,
               int store_dtype, void* Omega, void* Y);
/* Columns j0 <= j < j1 of the same Omega (the values nys_sketch draws for
 * them) and Y = Phi Omega for those columns only, (j1 - j0) x N each: the
 * probe columns are independent (Sec. III-C), so ranks that share a sketch
 * each draw and apply their own slice.  0 <= j0 < j1 <= ell, else
 * NYS_EINVAL. */
int nys_sketch_cols(nys_ctx* ctx, nys_op* op, int phi_kind, int ell, int j0, int j1, uint64_t seed,
                    int store_dtype, void* Omega, void* Y);

/* Nystrom factor U, S_hat (Algorithm 1 steps 3-8).  Caller-owned device
 * buffers: U (N x ell, dtype `dtype`: NYS_F32, NYS_F64 or NYS_BF16) and
 * S_hat (ell doubles, descending).  The library attaches small state of its
 * own (O(ell^2) device memory: U^T U of the stored U and the ell x ell matrix
 * that applies P^{-1}) to `priv`; release it with nys_precond_release.
 * nys_factor synchronises with the stream before returning and fills the
 * host fields marked "out".  It also runs nys_precond_setup(mu = 0,
 * sqrt_shift = 1). */
typedef struct nys_precond {
    void* U;
    double* S_hat;
    int64_t N;
    int ell;
    int dtype;
    double v;            /* out: final shift eps*||Omega||_F * 10^retries  */
    int chol_retries;    /* out                                            */
    double s_first;      /* out: S_hat[0]                                  */
    double s_last;       /* out: S_hat[ell-1]                              */
    double mu;           /* set by nys_precond_setup                       */
    int sqrt_shift;      /* set by nys_precond_setup                       */
    int ell_active;      /* out (setup): columns with d_i > 0, the only
                            ones P and P^{-1} read (d is non-increasing)   */
    void* priv;          /* library-owned; NULL before nys_factor          */
} nys_precond;

/* Omega, Y: N x ell in `in_dtype` (as written by nys_sketch).  eps is the
 * "machine accuracy" of Algorithm 1.  On Cholesky failure the shift is
 * multiplied by 10 and retried up to 8 times, then NYS_ENOTSPD.  The core is
 * symmetrised, (M + M^T)/2, before the Cholesky. */
int nys_factor(nys_ctx* ctx, const void* Omega, const void* Y, int in_dtype,
               int64_t N, int ell, double eps, nys_precond* out);
int nys_precond_release(nys_precond* pc);
/* Algorithm 1 steps 3-8 at the ell x ell level, from the Gram G2 of
 * [Omega | Y] (device, float64, 2 ell x 2 ell, row-major; only the blocks
 * Omega^T Omega, Omega^T Y, Y^T Y are read): the shift v = eps sqrt(trace
 * Omega^T Omega), the shifted Cholesky C of sym(Omega^T Y) + v Omega^T Omega
 * (retries as nys_factor), the eigen-decomposition V S^2 V^T of
 * C^{-1} Y_v^T Y_v C^{-T} = B^T B, S_hat (device, ell doubles, descending)
 * and W = C^{-T} V S^{-1} (device, ell x ell float64, row-major), so that
 * U = (Y + v Omega) W.  Ranks that each hold a slice of the pixels sum their
 * partial Grams (nys_gram) and call this on the sum; each then forms its rows
 * of U with nys_tall_gemm.  eig_f64 = 0 runs the rotations in float32 (as
 * nys_factor does for float32 / bf16 sketches).  v, retries (host, may be
 * NULL) receive the shift and the retry count.  Synchronises;
 * NYS_ENOTSPD as nys_factor. */
int nys_factor_gram(nys_ctx* ctx, const double* G2, int ell, double eps, int eig_f64, double* W,
                    double* S_hat, double* v, int* retries);
/* nys_precond_import with K = U^T U given (device, ell x ell float64) rather
 * than computed from pc->U: for a factor whose U holds only this rank's rows
 * (pc->N = local rows), K is the sum of the ranks' partial Grams.  Apply such
 * a factor with precond_partial / precond_finish.  Synchronises. */
int nys_precond_import_gram(nys_ctx* ctx, nys_precond* pc, const double* K, double mu, int sqrt_shift);
/* Adopt a factor the caller wrote into pc->U and pc->S_hat (N, ell, dtype
 * set; e.g. a preconditioner saved earlier): computes U^T U of the stored U,
 * the host copies s_first / s_last, and runs nys_precond_setup(mu,
 * sqrt_shift).  Synchronises. */
int nys_precond_import(nys_ctx* ctx, nys_precond* pc, double mu, int sqrt_shift);

/* ------------------------------------------------------ preconditioner -- */
/* Choose mu and the s_K <- sqrt(s_K) heuristic (Sec. III-B) and precompute
 * the weights d_i = max(0, (s_i + mu)/(s' + mu) - 1), s' = sqrt(s_K) or s_K,
 * of P = I + Ubar Ubar^T, Ubar = U diag(sqrt(d)) (the Sec. III-B rewrite of
 * Eq. RYPreconditioner), and M = diag(sqrt d) (I + Ubar^T Ubar)^{-1}
 * diag(sqrt d).  NYS_EDEGENERATE if s' + mu <= 0.  Synchronises. */
int nys_precond_setup(nys_ctx* ctx, nys_precond* pc, double mu, int sqrt_shift);

/* inverse = 0: out = P z = z + U diag(d) U^T z.
 * inverse = 1: out = P^{-1} z = z - U M U^T z.  This is the second line of
 * Eq. (RYPreconditioner) when U^T U = I, and the exact inverse of P for the
 * stored U otherwise (Woodbury), so P P^{-1} = I also when U is stored in
 * BF16.  z, out: batch*N of `dtype` (NYS_F32/NYS_F64); out == z allowed;
 * batches above 65535 images run in chunks of 65535 (scratch for one chunk). */
int precond_apply(nys_ctx* ctx, const nys_precond* pc, int inverse, int dtype,
                  const void* z, void* out, int batch);

/* precond_apply split in two for a factor whose U holds only this rank's
 * rows (pixel-sharded problems): precond_partial writes w[b] = U_r^T z_r[b]
 * (ell_active values per image, float64 for NYS_F64 data, float32
 * otherwise, device); the ranks sum w (an all-reduce of ell_active values per
 * image); precond_finish then writes out[b] = z[b] - U_r M w[b] (inverse = 1)
 * or z[b] + U_r diag(d) w[b], the rows of P^{-1} z or P z held by this rank.
 * Rows a multiple of the 16-byte vector width (8 bf16, 4 f32, 2 f64),
 * buffers 16-byte aligned, 1 <= batch <= 65535; NYS_EINVAL otherwise. */
int precond_partial(nys_ctx* ctx, const nys_precond* pc, int dtype, const void* z, void* w, int batch);
int precond_finish(nys_ctx* ctx, const nys_precond* pc, int inverse, int dtype, const void* w, const void* z,
                   void* out, int batch);

/* precond_apply for callers that cannot allocate device memory (no
 * cudaMalloc is allowed on their side: e.g. while another component captures
 * the stream into a CUDA graph, or under a fixed memory budget).  The paper
 * has no counterpart; this is a deployment variant of precond_apply with the
 * same arguments and results, computed by the plain kernels of
 * precond_apply's general path (not its vectorised ones), one image of the
 * batch at a time, over the active columns only.  Its scratch is one fixed
 * device array of NYS_NOALLOC_SCRATCH_BYTES (2 MiB) compiled into the
 * library, which every process that loads the library keeps on each GPU it
 * uses until exit.  Limit: (ceil(N/1024) * ell_active + ell_active) values of
 * the compute type (4 bytes for f32/bf16 factors, 8 for f64) must fit, e.g.
 * N = 512*512 with ell_active <= 2040 in f32; larger problems get NYS_EINVAL
 * (use precond_apply).  The call
 * allocates nothing.  Its first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the one array: calls whose kernels overlap on the
 * GPU (different streams, or several contexts) race and give wrong results;
 * calls issued in order on one stream are safe.  Nothing in the array needs
 * clearing: each call writes every entry it later reads. */
#define NYS_NOALLOC_SCRATCH_BYTES (2u * 1024u * 1024u)
int precond_apply_noalloc(nys_ctx* ctx, const nys_precond* pc, int inverse, int dtype,
                          const void* z, void* out, int batch);

/* ---------------------------------------------------------------- prox -- */
typedef struct nys_prox_info {
    int iterations;      /* Newton steps taken                 */
    int converged;       /* 1 if ||F|| reached the tolerance   */
    double residual;     /* final ||F(gamma)||                 */
} nys_prox_info;

/* Theorem 1 prox of tau ||.||_1 in the P metric (wavelet regulariser):
 * out = T_tau(s - Ubar gamma*) where gamma* solves
 * Ubar^T (s - T_tau(s - Ubar gamma)) + gamma = 0 by semi-smooth Newton.
 * pc == NULL gives the plain soft threshold.  gamma_io: device, ell doubles,
 * warm start in / solution out (may be NULL).  info (host, may be NULL) is
 * filled after an internal synchronisation. */
int prox_wavelet(nys_ctx* ctx, const nys_precond* pc, double tau, int dtype,
                 int64_t N, const void* s, void* out, double* gamma_io,
                 nys_prox_info* info);

/* Dual APG prox of lambda_bar ||L x||_{1,phi} in the P metric (Sec. III-B):
 * L = first differences with phi = 1 (prox_tv, Q: 2*N) or second differences
 * with the Schatten-1 norm (prox_hs, Q: 3*N as (q11, q12, q22) planes);
 * n_inner APG steps on the dual, warm-started from Q_io (in/out, caller
 * zeroes it before the first call).  pc == NULL gives P = I. */
int prox_tv(nys_ctx* ctx, const nys_precond* pc, double lambda_bar, int n_inner,
            int dtype, int n1, int n2, const void* s, void* out, void* Q_io);
int prox_hs(nys_ctx* ctx, const nys_precond* pc, double lambda_bar, int n_inner,
            int dtype, int n1, int n2, const void* s, void* out, void* Q_io);
/* The same dual APG for any mixed-norm regulariser of Eq. lpl1qMixedNorm:
 * reg = NYS_REG_TV, NYS_REG_ISOTV (Q: 2*N) or NYS_REG_HS, NYS_REG_HS2,
 * NYS_REG_HSINF (Q: 3*N).  The dual ball is that of l_{inf,psi},
 * 1/phi + 1/psi = 1 (Eq. mixedUnitNormBall), projected per pixel: clip
 * (TV), Euclidean scaling (isotropic TV), eigenvalue clip (HS_1), Frobenius
 * scaling with the cross term counted twice (HS_2), eigenvalues onto the l1
 * ball (HS_inf).  NYS_EINVAL for NYS_REG_WAVELET or an unknown reg. */
int prox_mixed(nys_ctx* ctx, const nys_precond* pc, int reg, double lambda_bar, int n_inner,
               int dtype, int n1, int n2, const void* s, void* out, void* Q_io);

/* ---------------------------------------------------------- Algorithm 2 -- */
/* Iteratively reweighted minimisation for the l_p - l_q problem of Eq.
 * lplqReg, min (1/p) sum |Ax - y|^p + (lambda/q) sum |(L x)_l^zeta|^q with L the
 * first differences (each of the two components its own element).  Outer
 * iteration k (Algorithm 2, Eqs. v:z:updating and WfWg:IRM): W_f =
 * |A x - y|_eps^{p-2}, W_g = |L x|_eps^{q-2} (|r|_eps = sqrt(r^2 + eps)), then
 * x solves (A^T W_f A + lambda L^T W_g L) x = A^T W_f y (Eq.
 * lplq:sub:updateX:linearEq) by conjugate gradients from the previous x,
 * preconditioned (ell > 0) with the Nystrom preconditioner of that matrix
 * built on the fly (Algorithm 1 on Omega drawn with seed + k, Eq.
 * RYPreconditioner with mu = 0).  CG stops at ||r|| <= cg_tol ||b||. */
typedef struct nys_irm_desc {
    double p;            /* data-term exponent, 0 < p <= 2                  */
    double q;            /* regulariser exponent, 0 < q <= 2                */
    double lambda;       /* >= 0                                            */
    double eps;          /* > 0                                             */
    int ell;             /* sketch size per outer iteration; 0 = plain CG   */
    int store_dtype;     /* sketch storage: NYS_BF16 or NYS_F32 for float32
                            operators, NYS_F64 for float64 ones             */
    uint64_t seed;
    double cg_tol;       /* > 0                                             */
    int cg_max;          /* >= 1                                            */
} nys_irm_desc;
typedef struct nys_irm_info {
    int cg_iters;        /* CG iterations of the outer iteration            */
    double residual;     /* ||r|| / ||b|| at exit                           */
    double rel_change;   /* ||x^k - x^{k-1}|| / ||x^k||                      */
} nys_irm_info;
typedef struct nys_irm nys_irm;
/* y: device, M values of the op dtype (copied).  x starts at 0.  The handle
 * keeps op and ctx; destroy it before the op. */
int nys_irm_create(nys_ctx* ctx, nys_op* op, const nys_irm_desc* desc, const void* y, nys_irm** out);
/* One outer iteration; synchronises the ctx stream once per CG iteration
 * (the stopping test).  info (host) may be NULL. */
int nys_irm_step(nys_irm* irm, nys_irm_info* info);
/* x (device, N values of the op dtype). */
int nys_irm_get_x(const nys_irm* irm, void* x);
/* x = 0 and the outer count (and so the probe seeds) restart. */
int nys_irm_reset(nys_irm* irm);
int nys_irm_destroy(nys_irm* irm);

/* ---------------------------------------------------------- Algorithm 3 -- */
typedef struct nys_solver_desc {
    int reg;             /* NYS_REG_*                                       */
    int fit;             /* NYS_FIT_L2 or NYS_FIT_HUBER                     */
    double lambda;       /* regularisation weight                           */
    double huber_delta;
    double alpha;        /* step size; <= 0: 1.02 x power-iteration estimate */
    int n_inner;         /* dual APG steps per prox (TV, HS)                */
    int power_iters;     /* power iterations for alpha (default 50)         */
    uint64_t power_seed;
    int no_graph;        /* 1: launch kernels one by one instead of replaying
                            the captured CUDA graph of an iteration          */
} nys_solver_desc;

/* WAPG (Algorithm 3) for min_x f(x) + lambda g(x) with operator op, data y
 * (device, M values, copied) and preconditioner pc (NULL = plain APG).  For
 * NYS_REG_WAVELET the variable is xbar = W x.  The solver owns x, u, t and
 * the dual/Newton warm starts; x^1 = u^1 = 0, t^0 = 1. */
int nys_solver_create(nys_ctx* ctx, nys_op* op, const nys_solver_desc* desc,
                      const void* y, const nys_precond* pc, nys_solver** solver);
int nys_solver_destroy(nys_solver* solver);
/* Run n_steps iterations of Algorithm 3 (asynchronous; graph-capturable). */
int pgd_step(nys_solver* solver, int n_steps);
/* Reset to x = u = 0, t = 1, zero warm starts (keeps alpha). */
int nys_solver_reset(nys_solver* solver);
/* Reset, and (if reestimate_alpha and the step size was not given) estimate
 * alpha again -- after the preconditioner was re-factored in place.
 * Synchronises when it estimates. */
int nys_solver_restart(nys_solver* solver, int reestimate_alpha);
/* Replace the data y (device, M values, copied) and reset the iterate. */
int nys_solver_set_data(nys_solver* solver, const void* y);
/* Copy the current iterate, in the image domain (W^T xbar for wavelets),
 * to x_out (device, N values of the op dtype). */
int nys_solver_get_x(nys_solver* solver, void* x_out);
/* Objective F(x) = f(x) + lambda g(x) at the current iterate (host, float64
 * accumulation): f = 1/2 ||A x - y||^2 or the Huber sum, g = anisotropic TV,
 * Hessian Schatten-1 or ||xbar||_1.  Synchronises. */
int nys_solver_objective(nys_solver* solver, double* F);
/* The step size in use (host).  Synchronises if it was estimated. */
int nys_solver_alpha(nys_solver* solver, double* alpha);

/* ------------------------------------------ differentiated unrolled solve -- */
/* Not in the paper: gradients of a truncated solve for learning lambda and
 * the blur kernel.  The map is K iterations of Algorithm 3 with the
 * anisotropic TV regulariser (quadratic data term), each prox the dual APG of
 * Sec. III-B with n_inner steps warm-started from the previous iteration's
 * dual, x^1 = u^1 = 0.  P and alpha are constants of the map. */
typedef struct nys_unroll nys_unroll;
typedef struct nys_unroll_desc {
    double lambda;       /* TV weight, > 0                                   */
    double alpha;        /* step size, > 0                                   */
    int K;               /* outer iterations, >= 1                           */
    int n_inner;         /* dual APG steps per prox, >= 0                    */
    int ckpt_every;      /* keep (x, u, Q) every ckpt_every iterations and
                            re-run each segment in the backward pass (0 = K) */
} nys_unroll_desc;

/* Allocates all device memory the forward and backward passes use: about
 * (5 + 4 ceil(K / ckpt_every) + 18) N + 2 M values plus ckpt_every (N + M +
 * 2 (n_inner + 1) N) for the segment record.  op must be f32 or f64 (the
 * dtype of every buffer below); pc (may be NULL: P = I) must stay alive and
 * unchanged while the handle is used. */
int nys_unroll_create(nys_ctx* ctx, nys_op* op, const nys_precond* pc,
                      const nys_unroll_desc* desc, nys_unroll** out);
int nys_unroll_destroy(nys_unroll* u);
/* x_out (device, N values; may be NULL) = x^{K+1} for data y (device, M
 * values, copied).  Keeps the checkpoints for nys_unroll_backward. */
int nys_unroll_forward(nys_unroll* u, const void* y, void* x_out);
/* Reverse pass of the last forward: for the cotangent xbar (device, N values)
 * of x^{K+1}, writes grads[0] = <xbar, d x / d lambda> and, for a blur
 * operator, grads[1 + a kw + b] = <xbar, d x / d h[a][b]> (grads: device,
 * float64, 1 + kh kw values).  NYS_EINVAL if no forward ran since the handle
 * was created or lambda changed. */
int nys_unroll_backward(nys_unroll* u, const void* xbar, double* grads);
/* Change lambda (invalidates the last forward). */
int nys_unroll_set_lambda(nys_unroll* u, double lambda);

/* -------------------------------------------------- batched unrolled solves -- */
/* Not in the paper: many unrolled solves (mixed sizes, operators and sketch
 * sizes) replayed as one CUDA graph.  items[i] and its operator must have
 * been created on item_ctx[i], whose stream must be its own (not ctx's);
 * ys[i] (M_i values), xs[i] (N_i), xbars[i] (N_i) are device buffers of the
 * item's dtype and grads[i] a device float64 buffer of 1 + kh kw values (as
 * nys_unroll_backward), all fixed for the life of the batch.  Creation runs
 * every item forward and backward once (synchronising), then captures the
 * two graphs: the batch stream forks to the item streams, which run
 * concurrently as branches of the graph, and joins them.  Not thread-safe. */
typedef struct nys_batch nys_batch;
int nys_batch_create(nys_ctx* ctx, int n, nys_unroll* const* items, nys_ctx* const* item_ctx,
                     const void* const* ys, void* const* xs, const void* const* xbars,
                     double* const* grads, nys_batch** out);
/* One graph launch on ctx's stream: every item's forward (xs <- x^{K+1}). */
int nys_batch_forward(nys_batch* b);
/* One graph launch: every item's reverse pass for its xbars (grads <- ...).
 * NYS_EINVAL before the first nys_batch_forward. */
int nys_batch_backward(nys_batch* b);
int nys_batch_destroy(nys_batch* b);

/* ------------------------------------------------------- dense products -- */
/* C (p x q, float64, row-major, device) = A^T B for tall operands A (N x p)
 * and B (N x q) stored as columns of N contiguous values (the layout of
 * Omega, Y and U): the Gram products of Algorithm 1 steps 5-7 and U^T U.
 * path 0: tcgen05 tensor cores for bf16 operands when q <= 256 and N is a
 * multiple of 8, else CUDA cores; 1: CUDA cores; 2: tensor cores or
 * NYS_EINVAL.  Float32 accumulation, splits summed in float64.
 * Synchronises (to report NYS_ETIMEOUT from a bounded pipeline wait). */
int nys_gram(nys_ctx* ctx, int dtype, const void* A, int p, const void* B, int q,
             int64_t N, double* C, int path);

/* out (q columns of N, out_dtype) = (A + alpha A2) W for tall A, A2 (k
 * columns of N, in_dtype; A2 may be NULL) and W (k x q float64, row-major,
 * device): with A = Y, A2 = Omega, alpha = v this is U = Y_v (C^{-T} V S^{-1})
 * of Algorithm 1 steps 6-7.  path as in nys_gram (tensor cores need bf16
 * inputs, A2 given, k = q <= 256, N a multiple of 8 and >= 128).
 * Synchronises. */
int nys_tall_gemm(nys_ctx* ctx, int in_dtype, const void* A, const void* A2, double alpha,
                  int64_t N, int k, const double* W, int q, int out_dtype, void* out, int path);

/* ---------------------------------------------------------- reductions -- */
/* *out (host) = ||a - b||_2 / ||b||_2 over n elements (b != 0), or ||a||_2
 * when b == NULL.  Synchronises. */
int nys_rel_err(nys_ctx* ctx, int dtype, int64_t n, const void* a, const void* b, double* out);

#ifdef __cplusplus
}
#endif
#endif /* NYS_H */
