// ell x ell dense kernels of Algorithm 1 (steps 3, 5, 7, 8) and of the
// preconditioner set-up.  All inputs come from float64 Gram matrices.
//
//   shift_chol   v = eps sqrt(trace(Omega^T Omega)) (= eps ||Omega||_F, step 3);
//                C = chol(sym(Omega^T Y) + v Omega^T Omega) (= chol(Omega^T Y_v),
//                step 5) with v <- 10 v retries; one CTA, float64.
//   form_H       H = Y_v^T Y_v = Y^T Y + v (Omega^T Y + Y^T Omega) + v^2 Omega^T Omega
//   tri_inv      C^{-1} for lower-triangular C, one warp per column
//   small_gemm   C = op(A) op(B) diag(colscale), float64
//   jacobi       cyclic Jacobi with the round-robin parallel ordering
//                (Golub & Van Loan, Sec. 8.5: sym.schur2 rotations, every
//                index in exactly one pair per round), one CTA, working type T
//   rayleigh     lambda_i = v_i^T G v_i / v_i^T v_i in float64
//   sort_eig     descending order of eigenpairs
//
// The float64 pipe of GB300 issues about two FMAs per clock per SM, so the
// Jacobi rotations run in float32 when the path's working type is float32;
// the eigenvalues are then Rayleigh quotients in float64, accurate to second
// order in the eigenvector error.
#include "internal.cuh"
#include "chol.cuh"

#include <cmath>
#include <cstdlib>

namespace nys {

// G2: (2 ell) x (2 ell) Gram of [Omega | Y] (row-major, ld = 2 ell).
// info[0] = status (0 ok, 1 not SPD), info[1] = v, info[2] = retries.
__global__ void __launch_bounds__(1024) shift_chol_kernel(const double* __restrict__ G2, int ell, double eps,
                                                          int max_retries, double* __restrict__ C,
                                                          double* __restrict__ info) {
    __shared__ int flag;
    __shared__ double sh[32];
    const int ld = 2 * ell;
    double tr = 0.0;
    for (int i = threadIdx.x; i < ell; i += blockDim.x) tr += G2[(size_t)i * ld + i];
    tr = block_sum(tr, sh);
    double v = eps * sqrt(tr);
    int r = 0;
    bool ok = false;
    for (; r <= max_retries; ++r) {
        for (int t = threadIdx.x; t < ell * ell; t += blockDim.x) {
            const int i = t / ell, j = t % ell;
            const double oy = 0.5 * (G2[(size_t)i * ld + ell + j] + G2[(size_t)j * ld + ell + i]);
            C[t] = oy + v * G2[(size_t)i * ld + j];
        }
        __syncthreads();
        ok = block_cholesky(C, ell, &flag);
        if (ok) break;
        v *= 10.0;
    }
    if (threadIdx.x == 0) {
        info[0] = ok ? 0.0 : 1.0;
        info[1] = v;
        info[2] = (double)(ok ? r : max_retries);
    }
}

// H = Y^T Y + v (Omega^T Y + Y^T Omega) + v^2 Omega^T Omega
__global__ void form_H_kernel(const double* __restrict__ G2, int ell, const double* __restrict__ info,
                              double* __restrict__ H) {
    const double v = info[1];
    const int ld = 2 * ell;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ell * ell; t += gridDim.x * blockDim.x) {
        const int i = t / ell, j = t % ell;
        const double yy = G2[(size_t)(ell + i) * ld + ell + j];
        const double oy = G2[(size_t)i * ld + ell + j] + G2[(size_t)j * ld + ell + i];
        const double oo = G2[(size_t)i * ld + j];
        H[t] = yy + v * oy + v * v * oo;
    }
}

// X = C^{-1} for lower-triangular C (n x n).  Block j (one warp) solves
// C x = e_j by forward substitution, with x in shared memory (the dependent
// chain of the substitution stays on chip) and rows of C read coalesced;
// column j of X is written at the end.  Dynamic shared memory: n doubles.
__global__ void tri_inv_kernel(const double* __restrict__ C, double* __restrict__ X, int n) {
    extern __shared__ __align__(16) double tx[];
    const int j = blockIdx.x;
    const int lane = threadIdx.x;
    if (lane == 0) tx[j] = 1.0 / C[(size_t)j * n + j];
    __syncwarp();
    for (int i = j + 1; i < n; ++i) {
        double s = 0.0;
        for (int k = j + lane; k < i; k += 32) s += C[(size_t)i * n + k] * tx[k];
        s = warp_sum(s);
        if (lane == 0) tx[i] = -s / C[(size_t)i * n + i];
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) X[(size_t)i * n + j] = i < j ? 0.0 : tx[i];
}

// C (m x n) = op(A) op(B) * colscale[j]  (row-major; op = transpose if flag)
__global__ void small_gemm_kernel(const double* __restrict__ A, int ta, const double* __restrict__ B, int tb, int m,
                                  int n, int k, const double* __restrict__ colscale, double* __restrict__ C) {
    __shared__ double As[16][17];
    __shared__ double Bs[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
    double acc = 0.0;
    for (int k0 = 0; k0 < k; k0 += 16) {
        const int ka = k0 + tx, kb = k0 + ty;
        // A(i, ka): ta ? A[ka][i] (A is k x m) : A[i][ka] (A is m x k)
        As[ty][tx] = (i < m && ka < k) ? (ta ? A[(size_t)ka * m + i] : A[(size_t)i * k + ka]) : 0.0;
        // B(kb, j): tb ? B[j][kb] (B is n x k) : B[kb][j] (B is k x n)
        Bs[ty][tx] = (kb < k && j < n) ? (tb ? B[(size_t)j * k + kb] : B[(size_t)kb * n + j]) : 0.0;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) acc = fma(As[ty][kk], Bs[kk][tx], acc);
        __syncthreads();
    }
    if (i < m && j < n) C[(size_t)i * n + j] = acc * (colscale ? colscale[j] : 1.0);
}

template <class T>
__global__ void copy_pad(const double* __restrict__ G, int ell, T* __restrict__ Gw, int n) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ell * ell; t += gridDim.x * blockDim.x) {
        const int i = t / ell, j = t % ell;
        Gw[(size_t)i * n + j] = (T)(0.5 * (G[t] + G[(size_t)j * ell + i]));
    }
}

// Jacobi eigensolver.  G: n x n (n even, the last index a zero pad when the
// real size is odd), overwritten by (nearly) diagonal; V: eigenvectors in
// columns.  arr holds the round-robin arrangement.
template <class T>
__global__ void __launch_bounds__(1024) jacobi_kernel(T* __restrict__ G, T* __restrict__ V, int n, int nreal,
                                                      int max_sweeps, double tol, int* __restrict__ sweeps_out,
                                                      const int* __restrict__ only_if_failed) {
    // runs only when the one-sided kernel reported a failed Cholesky
    if (only_if_failed && *only_if_failed == 0) return;
    __shared__ int arr[1024];
    __shared__ int arr2[1024];
    __shared__ int pp[512], qq[512];
    __shared__ T cs[512], sn[512];
    __shared__ double sh[32];
    const int h = n / 2;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) V[t] = (t / n == t % n) ? T(1) : T(0);
    for (int t = threadIdx.x; t < n; t += blockDim.x) arr[t] = t;
    __syncthreads();
    const T eps = sizeof(T) == 8 ? T(1e-15) : T(1e-7);
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double off = 0.0, dg = 0.0;
        for (int t = threadIdx.x; t < nreal * nreal; t += blockDim.x) {
            const int i = t / nreal, j = t % nreal;
            const double g = (double)G[(size_t)i * n + j];
            if (i == j) dg += g * g;
            else off += g * g;
        }
        off = block_sum(off, sh);
        dg = block_sum(dg, sh);
        if (off <= tol * tol * dg) break;
        for (int round = 0; round < n - 1; ++round) {
            for (int k = threadIdx.x; k < h; k += blockDim.x) {
                const int a = arr[k], b = arr[n - 1 - k];
                const int p = min(a, b), q = max(a, b);
                T c = T(1), s = T(0);
                if (q < nreal) {
                    const T apq = G[(size_t)p * n + q];
                    const T app = G[(size_t)p * n + p], aqq = G[(size_t)q * n + q];
                    if (fabs((double)apq) > (double)eps * sqrt(fabs((double)app * (double)aqq)) && apq != T(0)) {
                        const T tau = (aqq - app) / (T(2) * apq);
                        const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
                        c = T(1) / sqrt(T(1) + t * t);
                        s = t * c;
                    }
                }
                pp[k] = p;
                qq[k] = q;
                cs[k] = c;
                sn[k] = s;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < h * h; t += blockDim.x) {
                const int k1 = t / h, k2 = t % h;
                const int p1 = pp[k1], q1 = qq[k1], p2 = pp[k2], q2 = qq[k2];
                const T c1 = cs[k1], s1 = sn[k1], c2 = cs[k2], s2 = sn[k2];
                if (s1 == T(0) && s2 == T(0)) continue;
                T* gp = G + (size_t)p1 * n;
                T* gq = G + (size_t)q1 * n;
                const T xpp = gp[p2], xpq = gp[q2], xqp = gq[p2], xqq = gq[q2];
                const T rpp = c1 * xpp - s1 * xqp, rpq = c1 * xpq - s1 * xqq;
                const T rqp = s1 * xpp + c1 * xqp, rqq = s1 * xpq + c1 * xqq;
                T ypp = c2 * rpp - s2 * rpq, ypq = s2 * rpp + c2 * rpq;
                T yqp = c2 * rqp - s2 * rqq, yqq = s2 * rqp + c2 * rqq;
                if (k1 == k2) ypq = yqp = T(0);
                gp[p2] = ypp;
                gp[q2] = ypq;
                gq[p2] = yqp;
                gq[q2] = yqq;
            }
            for (int t = threadIdx.x; t < n * h; t += blockDim.x) {
                const int i = t / h, k = t % h;
                const T c = cs[k], s = sn[k];
                if (s == T(0)) continue;
                T* vr = V + (size_t)i * n;
                const T vp = vr[pp[k]], vq = vr[qq[k]];
                vr[pp[k]] = c * vp - s * vq;
                vr[qq[k]] = s * vp + c * vq;
            }
            // next arrangement: element 0 fixed, the others rotate by one
            for (int t = threadIdx.x; t < n; t += blockDim.x) arr2[t] = (t == 0) ? arr[0] : (t == 1 ? arr[n - 1] : arr[t - 1]);
            __syncthreads();
            for (int t = threadIdx.x; t < n; t += blockDim.x) arr[t] = arr2[t];
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) *sweeps_out = sweep;
}

// Jacobi with G held in shared memory (pitch n + 1).  V is not formed here:
// every round's rotations (pairs and (c, s)) are appended to a log in global
// memory, and rot_apply_kernel builds V = J_1 J_2 ... J_r afterwards with one
// warp per row of V (the rows are independent).  rounds_out = rounds logged.
template <class T>
__global__ void __launch_bounds__(1024) jacobi_smem_kernel(const T* __restrict__ Gin, int n, int nreal,
                                                           int max_sweeps, double tol, int2* __restrict__ logpq,
                                                           T* __restrict__ logcs, int* __restrict__ rounds_out,
                                                           int* __restrict__ sweeps_out,
                                                           const int* __restrict__ only_if_failed) {
    // runs only when the one-sided kernel reported a failed Cholesky
    if (only_if_failed && *only_if_failed == 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int h = n / 2;
    const int pitch = n + 1;
    T* G = reinterpret_cast<T*>(smem_raw);
    T* cs = G + (size_t)n * pitch;
    T* sn = cs + h;
    int* arr = reinterpret_cast<int*>(sn + h);
    int* arr2 = arr + n;
    int* pp = arr2 + n;
    int* qq = pp + h;
    __shared__ double sh[32];
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) G[(t / n) * pitch + t % n] = Gin[t];
    for (int t = threadIdx.x; t < n; t += blockDim.x) arr[t] = t;
    __syncthreads();
    const T eps = sizeof(T) == 8 ? T(1e-15) : T(1e-7);
    int sweep = 0, round_total = 0;
    __shared__ int nrot;   // rotations applied in the current sweep
    for (; sweep < max_sweeps; ++sweep) {
        double off = 0.0, dg = 0.0;
        for (int t = threadIdx.x; t < nreal * nreal; t += blockDim.x) {
            const int i = t / nreal, j = t % nreal;
            const double g = (double)G[i * pitch + j];
            if (i == j) dg += g * g;
            else off += g * g;
        }
        off = block_sum(off, sh);
        dg = block_sum(dg, sh);
        if (off <= tol * tol * dg) break;
        if (threadIdx.x == 0) nrot = 0;
        __syncthreads();
        for (int round = 0; round < n - 1; ++round, ++round_total) {
            for (int k = threadIdx.x; k < h; k += blockDim.x) {
                const int a = arr[k], b = arr[n - 1 - k];
                const int p = min(a, b), q = max(a, b);
                T c = T(1), s = T(0);
                if (q < nreal) {
                    const T apq = G[p * pitch + q];
                    const T app = G[p * pitch + p], aqq = G[q * pitch + q];
                    if (fabs((double)apq) > (double)eps * sqrt(fabs((double)app * (double)aqq)) && apq != T(0)) {
                        const T tau = (aqq - app) / (T(2) * apq);
                        const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
                        c = T(1) / sqrt(T(1) + t * t);
                        s = t * c;
                    }
                }
                pp[k] = p;
                qq[k] = q;
                cs[k] = c;
                sn[k] = s;
                if (s != T(0)) atomicAdd(&nrot, 1);
                logpq[(size_t)round_total * h + k] = make_int2(p, q);
                logcs[((size_t)round_total * h + k) * 2] = c;
                logcs[((size_t)round_total * h + k) * 2 + 1] = s;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < h * h; t += blockDim.x) {
                const int k1 = t / h, k2 = t % h;
                const T c1 = cs[k1], s1 = sn[k1], c2 = cs[k2], s2 = sn[k2];
                if (s1 == T(0) && s2 == T(0)) continue;
                const int p1 = pp[k1], q1 = qq[k1], p2 = pp[k2], q2 = qq[k2];
                T* gp = G + p1 * pitch;
                T* gq = G + q1 * pitch;
                const T xpp = gp[p2], xpq = gp[q2], xqp = gq[p2], xqq = gq[q2];
                const T rpp = c1 * xpp - s1 * xqp, rpq = c1 * xpq - s1 * xqq;
                const T rqp = s1 * xpp + c1 * xqp, rqq = s1 * xpq + c1 * xqq;
                T ypp = c2 * rpp - s2 * rpq, ypq = s2 * rpp + c2 * rpq;
                T yqp = c2 * rqp - s2 * rqq, yqq = s2 * rqp + c2 * rqq;
                if (k1 == k2) ypq = yqp = T(0);
                gp[p2] = ypp;
                gp[q2] = ypq;
                gq[p2] = yqp;
                gq[q2] = yqq;
            }
            for (int t = threadIdx.x; t < n; t += blockDim.x) arr2[t] = (t == 0) ? arr[0] : (t == 1 ? arr[n - 1] : arr[t - 1]);
            __syncthreads();
            for (int t = threadIdx.x; t < n; t += blockDim.x) arr[t] = arr2[t];
            __syncthreads();
        }
        // threshold criterion: a sweep without a single rotation has converged
        // to the working precision
        if (nrot == 0) {
            ++sweep;
            break;
        }
    }
    if (threadIdx.x == 0) {
        *sweeps_out = sweep;
        *rounds_out = round_total;
    }
}

// One-sided (Hestenes) Jacobi for the same eigenproblem: G = R^T R by an
// in-shared-memory Cholesky (upper R, column j at R + j * (n + 1)), then plane
// rotations of column pairs of R until all columns are mutually orthogonal;
// the accumulated rotation V holds the eigenvectors of G (R V has orthogonal
// columns, so V^T G V is diagonal).  Columns are contiguous in shared memory,
// so a pair's inner products and its update are stride-1.  The rotation log
// has the two-sided kernel's format.  status_out = 1 (and nothing logged) if
// the Cholesky meets a non-positive pivot, so that the two-sided kernel runs.
// 16-byte vectors of the working type (float4 / double2)
template <class T> struct JV;
template <> struct JV<float> { using type = float4; static constexpr int n = 4; };
template <> struct JV<double> { using type = double2; static constexpr int n = 2; };
__device__ __forceinline__ float vdot(float4 x, float4 y) { return x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w; }
__device__ __forceinline__ double vdot(double2 x, double2 y) { return x.x * y.x + x.y * y.y; }
__device__ __forceinline__ float4 vrot(float4 x, float4 y, float c, float s) {
    return make_float4(c * x.x - s * y.x, c * x.y - s * y.y, c * x.z - s * y.z, c * x.w - s * y.w);
}
__device__ __forceinline__ double2 vrot(double2 x, double2 y, double c, double s) {
    return make_double2(c * x.x - s * y.x, c * x.y - s * y.y);
}

// column pitch of R: a whole number of 16-byte vectors (the rows beyond n are
// zero), plus one vector in shared memory to spread the columns over banks
__host__ __device__ inline int jac_pitch(int n, bool global) { return ((n + 3) & ~3) + (global ? 0 : 4); }

template <class T, bool GLOBAL>
__global__ void __launch_bounds__(1024) jacobi_1s_kernel(const T* __restrict__ Gin, T* __restrict__ Rg, int n, int nreal,
                                                         int max_sweeps, int2* __restrict__ logpq,
                                                         T* __restrict__ logcs, int* __restrict__ rounds_out,
                                                         int* __restrict__ sweeps_out, int* __restrict__ status_out) {
    using VT = typename JV<T>::type;
    constexpr int VW = JV<T>::n;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int h = n / 2;
    // column j at R + j * pitch: shared memory with the Cholesky done here, or
    // global memory holding the factor written by chol_upper_kernel (which
    // also set *status_out)
    const int pitch = jac_pitch(n, GLOBAL);
    T* R = GLOBAL ? Rg : reinterpret_cast<T*>(smem_raw);
    T* nrm = GLOBAL ? reinterpret_cast<T*>(smem_raw) : R + (size_t)n * pitch;   // n column norms
    T* rowk = nrm + n;                                                          // n (Cholesky row)
    __shared__ int bad;
    if (GLOBAL) {
        if (*status_out != 0) return;
    } else {
        // load G (symmetric) into R as column-major, pad index -> identity, pad rows -> 0
        for (int t = threadIdx.x; t < n * pitch; t += blockDim.x) {
            const int j = t / pitch, i = t % pitch;
            T g = T(0);
            if (i < n) {
                g = Gin[(size_t)i * n + j];
                if (i >= nreal || j >= nreal) g = (i == j) ? T(1) : T(0);
            }
            R[t] = g;
        }
        if (threadIdx.x == 0) bad = 0;
        __syncthreads();
        // in-place Cholesky, upper factor: R(k, j) for j >= k (column j holds rows 0..j)
        for (int k = 0; k < n; ++k) {
            if (threadIdx.x == 0) {
                const T d = R[k * pitch + k];
                if (!(d > T(0))) bad = 1;
                else R[k * pitch + k] = sqrt(d);
            }
            __syncthreads();
            if (bad) break;
            const T rkk = R[k * pitch + k];
            for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) {   // row k, columns j > k
                const T v = R[j * pitch + k] / rkk;
                R[j * pitch + k] = v;
                rowk[j] = v;
            }
            __syncthreads();
            // trailing update R(i, j) -= R(k, i) R(k, j), i <= j, rows fastest
            const int m = n - k - 1;
            for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
                const int j = k + 1 + t / m, i = k + 1 + t % m;
                if (i <= j) R[j * pitch + i] -= rowk[i] * rowk[j];
            }
            __syncthreads();
        }
        if (bad) {
            if (threadIdx.x == 0) *status_out = 1;
            return;
        }
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            const int i = t % n, j = t / n;   // zero the strict lower part
            if (i > j) R[j * pitch + i] = T(0);
        }
    }
    __syncthreads();
    // Threshold: a pair counts as orthogonal once |x.y| <= tol sqrt(|x|^2 |y|^2)
    // with tol = sqrt(n) eps; eigenvalues are recomputed afterwards in FP64 from
    // Rayleigh quotients, so this bounds only the eigenvector accuracy.
    const T tol = (sizeof(T) == 8 ? T(2.2e-16) : T(1.2e-7)) * sqrt(T(n));
    // gs threads per column pair (a power of two <= 32), every pair of a round
    // in flight at once; pairs by the circle method: player n-1 is fixed,
    // players 0..n-2 rotate, round r pairs (n-1, r) and (r+k, r-k) mod (n-1).
    // Column norms are kept up to date (|x'|^2 = |x|^2 - t c, |y'|^2 =
    // |y|^2 + t c for the rotation below) and recomputed at every sweep, so a
    // pair needs one inner product; columns move as 16-byte vectors.
    int gs = 32;
    while (gs > 1 && gs * h > (int)blockDim.x) gs >>= 1;
    const int ngroups = blockDim.x / gs;
    const int g = threadIdx.x / gs, gl = threadIdx.x % gs;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int nv = pitch / VW;   // vectors per column (pad rows are zero)
    const int m1 = n - 1;
    int sweep = 0, round_total = 0;
    for (; sweep < max_sweeps; ++sweep) {
        for (int j = warp; j < n; j += nwarps) {
            const VT* wj = reinterpret_cast<const VT*>(R + (size_t)j * pitch);
            T a = T(0);
            for (int v = lane; v < nv; v += 32) {
                const VT x = wj[v];
                a += vdot(x, x);
            }
            a = warp_sum(a);
            if (lane == 0) nrm[j] = a;
        }
        __syncthreads();
        int rotated = 0;
        for (int round = 0; round < m1; ++round, ++round_total) {
            for (int k0 = 0; k0 < h; k0 += ngroups) {
                const int k = k0 + g;
                const bool active = k < h;
                int p = 0, q = 1;
                if (active) {
                    const int u = (k == 0) ? m1 : (round + k) % m1;
                    const int w = (k == 0) ? round : (round - k + m1) % m1;
                    p = min(u, w);
                    q = max(u, w);
                }
                VT* wp = reinterpret_cast<VT*>(R + (size_t)p * pitch);
                VT* wq = reinterpret_cast<VT*>(R + (size_t)q * pitch);
                T c = T(0);
                if (active) {
#pragma unroll 4
                    for (int v = gl; v < nv; v += gs) c += vdot(wp[v], wq[v]);
                }
                for (int o = gs >> 1; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                if (!active) continue;
                const T a = nrm[p], b = nrm[q];
                T cs = T(1), sn = T(0);
                if (q < nreal && c != T(0) && fabs(c) > tol * sqrt(a * b)) {
                    const T zeta = (b - a) / (T(2) * c);
                    const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
                    cs = T(1) / sqrt(T(1) + t * t);
                    sn = t * cs;
#pragma unroll 4
                    for (int v = gl; v < nv; v += gs) {
                        const VT x = wp[v], y = wq[v];
                        wp[v] = vrot(x, y, cs, sn);
                        wq[v] = vrot(y, x, cs, -sn);   // sn x + cs y
                    }
                    if (gl == 0) {
                        nrm[p] = a - t * c;
                        nrm[q] = b + t * c;
                    }
                    rotated = 1;
                }
                if (gl == 0) {
                    const size_t e = (size_t)round_total * h + k;
                    logpq[e] = make_int2(p, q);
                    logcs[e * 2] = cs;
                    logcs[e * 2 + 1] = sn;
                }
            }
            __syncthreads();
        }
        if (!__syncthreads_or(rotated)) {
            ++sweep;
            break;
        }
    }
    if (threadIdx.x == 0) {
        *sweeps_out = sweep;
        *rounds_out = round_total;
        *status_out = 0;
    }
}

// Set-up of the global-memory one-sided Jacobi: work (n x n float64) = G
// padded with the identity, its float64 Cholesky L (one CTA), and R = L^T in
// the working type, column-major with pitch jac_pitch(n, true) (column j of R
// is row j of L, zero-padded).
// *status = 1 if a pivot is not positive; *rounds = 0 until the sweeps log.
template <class T>
__global__ void __launch_bounds__(1024) chol_upper_kernel(const double* __restrict__ G, int ell, int n,
                                                          double* __restrict__ work, T* __restrict__ R,
                                                          int* __restrict__ status, int* __restrict__ rounds) {
    __shared__ int flag;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int i = t / n, j = t % n;
        work[t] = (i < ell && j < ell) ? G[(size_t)i * ell + j] : (i == j ? 1.0 : 0.0);
    }
    if (threadIdx.x == 0) *rounds = 0;
    __syncthreads();
    const bool ok = block_cholesky(work, n, &flag);
    if (threadIdx.x == 0) *status = ok ? 0 : 1;
    if (!ok) return;
    const int pitch = jac_pitch(n, true);
    for (int t = threadIdx.x; t < n * pitch; t += blockDim.x) {
        const int j = t / pitch, i = t % pitch;
        R[t] = (i <= j && i < n) ? (T)work[(size_t)j * n + i] : T(0);
    }
}

// V[i][:] = e_i J_1 ... J_r, one warp per row (eight rows per CTA); pairs of
// a round are disjoint.  The log is staged through shared memory rch rounds
// at a time by the whole CTA, so the sequential rounds wait on shared-memory
// latency instead of global-memory latency.
template <class T>
__global__ void __launch_bounds__(256) rot_apply_kernel(const int2* __restrict__ logpq, const T* __restrict__ logcs,
                                                        const int* __restrict__ rounds, int n, int RCH,
                                                        T* __restrict__ V) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int h = n / 2;
    const int i = blockIdx.x * 8 + warp;
    T* rows = reinterpret_cast<T*>(smem_raw);              // 8 x n
    T* scs = rows + 8 * (size_t)n;                         // RCH x h x 2
    int2* spq = reinterpret_cast<int2*>(scs + (size_t)RCH * h * 2);   // RCH x h
    T* row = rows + (size_t)warp * n;
    for (int j = lane; j < n; j += 32) row[j] = (j == i) ? T(1) : T(0);
    const int R = *rounds;
    for (int r0 = 0; r0 < R; r0 += RCH) {
        const int nr = min(RCH, R - r0);
        __syncthreads();
        for (int t = threadIdx.x; t < nr * h; t += blockDim.x) {
            spq[t] = logpq[(size_t)r0 * h + t];
            scs[2 * t] = logcs[((size_t)r0 * h + t) * 2];
            scs[2 * t + 1] = logcs[((size_t)r0 * h + t) * 2 + 1];
        }
        __syncthreads();
        if (i < n) {
            for (int r = 0; r < nr; ++r) {
                for (int k = lane; k < h; k += 32) {
                    const T s = scs[2 * (r * h + k) + 1];
                    if (s == T(0)) continue;
                    const T c = scs[2 * (r * h + k)];
                    const int2 pq = spq[r * h + k];
                    const T vp = row[pq.x], vq = row[pq.y];
                    row[pq.x] = c * vp - s * vq;
                    row[pq.y] = s * vp + c * vq;
                }
                __syncwarp();
            }
        }
    }
    if (i < n)
        for (int j = lane; j < n; j += 32) V[(size_t)i * n + j] = row[j];
}

// lambda_i = v_i^T G v_i / (v_i^T v_i), G float64 (ld = ell), V (ld = n) of T.
template <class T>
__global__ void rayleigh_kernel(const double* __restrict__ G, const T* __restrict__ V, int ell, int n,
                                double* __restrict__ lam) {
    __shared__ double sh[32];
    const int i = blockIdx.x;
    double num = 0.0, den = 0.0;
    for (int r = threadIdx.x; r < ell; r += blockDim.x) {
        const double vr = (double)V[(size_t)r * n + i];
        double gv = 0.0;
        for (int c = 0; c < ell; ++c) gv += G[(size_t)r * ell + c] * (double)V[(size_t)c * n + i];
        num += vr * gv;
        den += vr * vr;
    }
    num = block_sum(num, sh);
    den = block_sum(den, sh);
    if (threadIdx.x == 0) lam[i] = num / den;
}

// sort eigenpairs descending; Vout (ell x ell float64, column k = k-th
// eigenvector), S2 = sorted eigenvalues, S_hat = max(0, S2 - v), scale = 1/sqrt(S2)
template <class T>
__global__ void sort_eig_kernel(const double* __restrict__ lam, const T* __restrict__ V, int ell, int n,
                                const double* __restrict__ info, double* __restrict__ Vout,
                                double* __restrict__ S_hat, double* __restrict__ scale) {
    const double v = info[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ell; i += gridDim.x * blockDim.x) {
        const double li = lam[i];
        int rank = 0;
        for (int j = 0; j < ell; ++j) {
            const double lj = lam[j];
            rank += (lj > li) || (lj == li && j < i);
        }
        S_hat[rank] = fmax(0.0, li - v);
        scale[rank] = li > 0.0 ? 1.0 / sqrt(li) : 0.0;
        for (int r = 0; r < ell; ++r) Vout[(size_t)r * ell + rank] = (double)V[(size_t)r * n + i];
    }
}

// d_i = max(0, (s_i + mu)/(s' + mu) - 1), s' = sqrt(s_K) or s_K; sqrt(d)
__global__ void weights_kernel(const double* __restrict__ S_hat, int ell, double mu, int sqrt_shift,
                               double* __restrict__ d, double* __restrict__ sqd, float* __restrict__ d32) {
    const double sk = S_hat[ell - 1];
    const double sref = sqrt_shift ? sqrt(fmax(sk, 0.0)) : sk;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ell; i += gridDim.x * blockDim.x) {
        const double di = fmax(0.0, (S_hat[i] + mu) / (sref + mu) - 1.0);
        d[i] = di;
        sqd[i] = sqrt(di);
        d32[i] = (float)di;
    }
}

// A (eff x eff) = I + diag(sqd) K diag(sqd) on the leading eff x eff block of K (ld = ldk)
__global__ void form_A_kernel(const double* __restrict__ K, int ldk, const double* __restrict__ sqd, int eff,
                              double* __restrict__ A) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < eff * eff; t += gridDim.x * blockDim.x) {
        const int i = t / eff, j = t % eff;
        A[t] = (i == j ? 1.0 : 0.0) + sqd[i] * 0.5 * (K[(size_t)i * ldk + j] + K[(size_t)j * ldk + i]) * sqd[j];
    }
}

__global__ void chol_kernel(double* __restrict__ A, int n, double* __restrict__ info) {
    __shared__ int flag;
    const bool ok = block_cholesky(A, n, &flag);
    if (threadIdx.x == 0) info[3] = ok ? 0.0 : 1.0;
}

// M (ell x ell) = diag(sqd) Ainv diag(sqd) on the leading eff x eff block
// (Ainv has ld = eff), zero elsewhere; also a float copy
__global__ void form_M_kernel(const double* __restrict__ Ainv, const double* __restrict__ sqd, int ell, int eff,
                              double* __restrict__ M, float* __restrict__ M32) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ell * ell; t += gridDim.x * blockDim.x) {
        const int i = t / ell, j = t % ell;
        const double m = (i < eff && j < eff) ? sqd[i] * Ainv[(size_t)i * eff + j] * sqd[j] : 0.0;
        M[t] = m;
        M32[t] = (float)m;
    }
}

// ---------------------------------------------------------------- host ---
int launch_small_gemm(nys_ctx* ctx, const double* A, int ta, const double* B, int tb, int m, int n, int k,
                      const double* colscale, double* C) {
    dim3 grid((n + 15) / 16, (m + 15) / 16);
    small_gemm_kernel<<<grid, 256, 0, ctx->stream>>>(A, ta, B, tb, m, n, k, colscale, C);
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

// Eigen-decomposition of the symmetric ell x ell float64 matrix G:
// Vout (ell x ell, columns sorted by descending eigenvalue), S_hat, scale.
// `work` provides 2 n^2 + n doubles (the float path: n^2 floats each for the
// padded copy, V and the cluster kernel's R, and n doubles).  `use_f32` picks
// the Jacobi type.
int sym_eig(nys_ctx* ctx, const double* G, int ell, bool use_f32, const double* info, void* work, double* Vout,
            double* S_hat, double* scale, int* sweeps_dev) {
    const int n = (ell + 1) & ~1;
    if (n > 1024) return fail(ctx, NYS_EINVAL, "sketch size above 1024 is not supported");
    cudaStream_t s = ctx->stream;
    auto run = [&](auto* tag) -> int {
        using T = std::remove_pointer_t<decltype(tag)>;
        T* Gw = (T*)work;
        T* V = Gw + (size_t)n * n;
        double* lam = (double*)(V + (size_t)n * n);
        // padded copy in the working type
        NYS_CK(ctx, cudaMemsetAsync(Gw, 0, sizeof(T) * n * n, s));
        copy_pad<T><<<64, 256, 0, s>>>(G, ell, Gw, n);
        NYS_LAUNCH_CK(ctx);
        // sweep cap: 30 (float64) or 15 (float32) unless NYS_EIG_SWEEPS sets it
        static const int env_sweeps = [] {
            const char* e = getenv("NYS_EIG_SWEEPS");
            const int v = e ? atoi(e) : 0;
            return v > 0 && v <= 100 ? v : 0;
        }();
        const int max_sweeps = env_sweeps ? env_sweeps : (sizeof(T) == 8 ? 30 : 15);
        const double tol = sizeof(T) == 8 ? 1e-14 : 2e-7;
        const int h = n / 2;
        int* status_dev = sweeps_dev + 2;
        if (sizeof(T) == 4) {
            // float32 sketches of 64..448 columns: the cluster kernel (Cholesky
            // and one-sided Jacobi spread over 8 or 16 SMs, V formed in place);
            // the two-sided kernel runs instead if its Cholesky fails
            // R's copy for the back substitution after lam: the work area holds
            // 2 n^2 doubles + n, the float path uses n^2 + n^2 floats + n doubles
            float* Rsave = (float*)(lam + n);
            const int stc = jacobi_cluster(ctx, G, ell, max_sweeps, (float*)V, n, Rsave, sweeps_dev, status_dev);
            if (stc == NYS_OK) {
                jacobi_kernel<T><<<1, 1024, 0, s>>>(Gw, V, n, ell, max_sweeps, tol, sweeps_dev, status_dev);
                NYS_LAUNCH_CK(ctx);
                rayleigh_kernel<T><<<ell, 128, 0, s>>>(G, V, ell, n, lam);
                NYS_LAUNCH_CK(ctx);
                sort_eig_kernel<T><<<(ell + 127) / 128, 128, 0, s>>>(lam, V, ell, n, info, Vout, S_hat, scale);
                NYS_LAUNCH_CK(ctx);
                return NYS_OK;
            }
            if (stc != NYS_EINVAL) return stc;
        }
        const size_t smem = sizeof(T) * ((size_t)n * (n + 1) + 2 * (size_t)h) + sizeof(int) * (2 * (size_t)n + 2 * h + 4) + 64;
        const size_t smem1 = sizeof(T) * ((size_t)n * jac_pitch(n, false) + 2 * (size_t)n) + 64;
        // both kernels of the shared-memory path must fit (leaving room for
        // their static shared memory)
        const bool in_smem = smem + 1024 <= 227 * 1024 && smem1 + 1024 <= 227 * 1024;
        // rotations are logged and V is built by many CTAs (rot_apply)
        int st;
        const size_t rounds = (size_t)max_sweeps * (n - 1);
        auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
        const size_t logb = al(rounds * h * (sizeof(int2) + 2 * sizeof(T)));
        const size_t extra =
            in_smem ? 0 : al((size_t)n * n * sizeof(double)) + al((size_t)n * jac_pitch(n, true) * sizeof(T));
        char* lg = (char*)scratch(ctx, SLOT_EIG, logb + extra + 64, &st);
        if (st) return st;
        int2* logpq = (int2*)lg;
        T* logcs = (T*)(lg + rounds * h * sizeof(int2));
        int* rounds_dev = sweeps_dev + 1;
        // one-sided Jacobi on the Cholesky factor of G; the two-sided kernel runs
        // instead (decided on the device) if that Cholesky fails
        if (in_smem) {
            if (int st2 = smem_optin(ctx, (const void*)jacobi_smem_kernel<T>, smem)) return st2;
            if (int st2 = smem_optin(ctx, (const void*)jacobi_1s_kernel<T, false>, smem1)) return st2;
            jacobi_1s_kernel<T, false><<<1, 1024, smem1, s>>>(Gw, nullptr, n, ell, max_sweeps, logpq, logcs,
                                                              rounds_dev, sweeps_dev, status_dev);
            NYS_LAUNCH_CK(ctx);
            jacobi_smem_kernel<T><<<1, 1024, smem, s>>>(Gw, n, ell, max_sweeps, tol, logpq, logcs, rounds_dev,
                                                        sweeps_dev, status_dev);
            NYS_LAUNCH_CK(ctx);
        } else {
            // too large for shared memory: float64 Cholesky of G, then the
            // one-sided sweeps on R held in global memory (L2-resident)
            double* w64 = (double*)(lg + logb);
            T* Rg = (T*)(lg + logb + al((size_t)n * n * sizeof(double)));
            chol_upper_kernel<T><<<1, 1024, 0, s>>>(G, ell, n, w64, Rg, status_dev, rounds_dev);
            NYS_LAUNCH_CK(ctx);
            jacobi_1s_kernel<T, true><<<1, 1024, 2 * (size_t)n * sizeof(T), s>>>(nullptr, Rg, n, ell, max_sweeps, logpq,
                                                                                  logcs, rounds_dev, sweeps_dev,
                                                                                  status_dev);
            NYS_LAUNCH_CK(ctx);
        }
        // staged rounds per pass of rot_apply: as many as fit in 96 KB
        const size_t per_round = (size_t)h * (2 * sizeof(T) + sizeof(int2));
        const int rch = (int)std::max<size_t>(1, std::min<size_t>(32, (96 * 1024) / per_round));
        const size_t rsm = 8 * (size_t)n * sizeof(T) + (size_t)rch * per_round;
        if (int st2 = smem_optin(ctx, (const void*)rot_apply_kernel<T>, rsm)) return st2;
        rot_apply_kernel<T><<<(n + 7) / 8, 256, rsm, s>>>(logpq, logcs, rounds_dev, n, rch, V);
        NYS_LAUNCH_CK(ctx);
        if (!in_smem) {
            // two-sided fallback in global memory (overwrites V) if the Cholesky failed
            jacobi_kernel<T><<<1, 1024, 0, s>>>(Gw, V, n, ell, max_sweeps, tol, sweeps_dev, status_dev);
            NYS_LAUNCH_CK(ctx);
        }
        rayleigh_kernel<T><<<ell, 128, 0, s>>>(G, V, ell, n, lam);
        NYS_LAUNCH_CK(ctx);
        sort_eig_kernel<T><<<(ell + 127) / 128, 128, 0, s>>>(lam, V, ell, n, info, Vout, S_hat, scale);
        NYS_LAUNCH_CK(ctx);
        return NYS_OK;
    };
    return use_f32 ? run((float*)nullptr) : run((double*)nullptr);
}

}  // namespace nys
