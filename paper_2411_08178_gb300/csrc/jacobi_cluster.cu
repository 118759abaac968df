// Eigen-decomposition of the ell x ell Gram G = B^T B of Algorithm 1 step 7 on
// a thread-block cluster: one-sided (Hestenes) Jacobi on the Cholesky factor
// R (G = R^T R), float32, for 64 <= ell <= 448.
//
// The columns of R are cut into 2C blocks of b columns; CTA c of the
// cluster holds two of them in shared memory (its two "seats").  The
// rotations are not accumulated: the sweeps turn R into R V (orthogonal
// columns) and V = R^{-1} (R V) is recovered afterwards by back substitution
// against a copy of R saved before the sweeps, so that a sub-round and a
// move between CTAs carry one float per row instead of two.
//   Cholesky   right-looking by panels (one block per panel): the panel's
//              owner factors its b x b diagonal block, every CTA solves for
//              the panel's rows of its own later columns, then updates its
//              columns with the panel's rows gathered from the other CTAs
//              (distributed shared memory); two cluster barriers per panel.
//   sweeps     one sweep pairs every column with every other once: a CTA
//              rotates every pair between its two blocks (b sub-rounds of b
//              disjoint pairs, one warp per pair), and in the first block
//              round also the pairs inside each block; then the blocks move
//              to the next seats of a round-robin tournament over the 2C
//              seats (seat 0 fixed, the others shift by one), copied from the
//              neighbouring CTAs' shared memory, and the next block round
//              starts.  2C - 1 block rounds per sweep; the sweeps stop when
//              no pair needed a rotation or every pair's |x . y| / (|x| |y|)
//              was below stop2^(1/2) (cluster-wide vote), or after
//              max_sweeps.
//   output     R V (row-major, ld = ldv): column idx is the rotated column
//              that started as column idx of R; jc_backsolve_kernel turns it
//              into V (unit columns), V^T G V diagonal.
// Every CTA runs the same sequence of cluster barriers (uniform control
// flow, no spin waits).  A non-positive Cholesky pivot sets *status_out = 1
// and writes nothing else, so that the caller's two-sided kernel runs.
#include "internal.cuh"
#include "chol_panel.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace nys {
namespace {

constexpr int JC_THREADS = 512;   // 16 warps: one per pair of a sub-round (b <= 16)

template <int C>
__global__ void __launch_bounds__(JC_THREADS, 1)
    jacobi_cluster_kernel(const double* __restrict__ G, int nreal, int b, int max_sweeps, float* __restrict__ V,
                          int ldv, float* __restrict__ Rsave, float stop2, int* __restrict__ sweeps_out,
                          int* __restrict__ status_out) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int npad = 2 * C * b;
    const int col_len = npad;
    const int slot_len = b * col_len;
    extern __shared__ __align__(16) float jc_smem[];
    float* buf = jc_smem;                         // [4][b][npad]: cur seat 0, cur seat 1, next seat 0, next seat 1
    float* nrm = buf + 4 * (size_t)slot_len;      // [4][b]
    int* idx = reinterpret_cast<int*>(nrm + 4 * b);   // [4][b]
    __shared__ int bad_flag, rot_flag, rmax_bits;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // seats: CTA c holds seats c and 2C - 1 - c; block k starts in seat k
    int cur = 0;                                  // buffers cur, cur + 1 are the current seats
    auto seat_buf = [&](int which) { return buf + (size_t)which * slot_len; };
    const int blk[2] = {rank, 2 * C - 1 - rank};
    for (int s = 0; s < 2; ++s)
        for (int c = threadIdx.x; c < b; c += blockDim.x) idx[s * b + c] = blk[s] * b + c;
    // load G (padded with the identity), columns of the two blocks
    for (int s = 0; s < 2; ++s) {
        float* sb = seat_buf(s);
        for (int t = threadIdx.x; t < b * npad; t += blockDim.x) {
            const int c = t / npad, i = t - c * npad;
            const int j = blk[s] * b + c;
            float g;
            if (i < nreal && j < nreal) g = (float)G[(size_t)i * nreal + j];
            else g = (i == j) ? 1.0f : 0.0f;
            sb[(size_t)c * col_len + i] = g;
        }
    }
    if (threadIdx.x == 0) bad_flag = 0;
    // the next-seat buffers serve as staging during the Cholesky
    float* stage = seat_buf(2);
    cluster.sync();

    // ---------------------------------------------------------- Cholesky --
    for (int k = 0; k < 2 * C; ++k) {
        const int owner = k < C ? k : 2 * C - 1 - k;
        const int oseat = k < C ? 0 : 1;
        const int p0 = k * b;                      // first column (and row) of the panel
        if (rank == owner) {
            // the b x b diagonal block by one warp (b <= 16, registers and shuffles)
            if (warp == 0) {
                float* pb = seat_buf(oseat);
                const bool ok = warp_chol_block<float>([&](int c) { return pb + (size_t)c * col_len; }, p0, b);
                if (!ok && lane == 0) bad_flag = 1;
            }
            __syncthreads();
            // a failed pivot: tell every CTA (their own copy of the flag), so
            // that all leave after the same barrier and no CTA reads the
            // shared memory of one that has left
            if (bad_flag && threadIdx.x < C) *cluster.map_shared_rank(&bad_flag, (int)threadIdx.x) = 1;
        }
        cluster.sync();
        if (bad_flag) {
            if (rank == 0 && threadIdx.x == 0) *status_out = 1;
            return;
        }
        // the panel's diagonal block R_PP (b x b, upper) from its owner
        {
            const float* ob = cluster.map_shared_rank(seat_buf(oseat), owner);
            for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
                const int c = e / b, i = e - c * b;
                stage[e] = ob[(size_t)c * col_len + p0 + i];   // stage[c b + i] = R(p0 + i, p0 + c)
            }
        }
        __syncthreads();
        // rows of the panel in my later columns: solve R_PP^T x = g (forward
        // substitution), one thread per column (a chain of b^2 / 2 FMAs is
        // shorter than b rounds of warp reductions)
        for (int cc = threadIdx.x; cc < 2 * b; cc += blockDim.x) {
            const int s = cc / b, c = cc - s * b;
            if (blk[s] <= k) continue;
            panel_forward_subst(seat_buf(s) + (size_t)c * col_len, stage, p0, b);
        }
        cluster.sync();
        // gather the panel's rows of every column after the panel: stage[i][m] = R(p0 + i, m)
        const int m0 = p0 + b;
        const int nm = npad - m0;
        if (nm > 0) {
            for (int e = threadIdx.x; e < b * nm; e += blockDim.x) {
                const int m = m0 + e / b, i = e - (e / b) * b;
                const int kb = m / b, c = m - kb * b;
                const int orank = kb < C ? kb : 2 * C - 1 - kb, os = kb < C ? 0 : 1;
                const float* ob = cluster.map_shared_rank(seat_buf(os), orank);
                stage[(size_t)b * b + (size_t)(m - m0) * b + i] = ob[(size_t)c * col_len + p0 + i];
            }
            __syncthreads();
            // trailing update of my later columns: R(i, j) -= sum_t R(p0 + t, i) R(p0 + t, j), m0 <= i <= j
            for (int s = 0; s < 2; ++s) {
                if (blk[s] <= k) continue;
                float* sb = seat_buf(s);
                const float* rows = stage + (size_t)b * b;
                for (int e = threadIdx.x; e < b * npad; e += blockDim.x) {
                    const int c = e / npad, i = e - c * npad;
                    const int j = blk[s] * b + c;
                    if (i < m0 || i > j) continue;
                    float* col = sb + (size_t)c * col_len;
                    float acc = 0.0f;
                    for (int t = 0; t < b; ++t) acc += rows[(size_t)(i - m0) * b + t] * col[p0 + t];
                    col[i] -= acc;
                }
            }
        }
        // the next panel's owner reads and writes only its own columns and
        // rows of later panels; the others read this panel's rows, which are final
        __syncthreads();
    }
    // R upper triangular (the strict lower parts still hold G); a copy of its
    // nreal x nreal part (column-major, ld nreal) for the back substitution
    for (int s = 0; s < 2; ++s) {
        float* sb = seat_buf(s);
        for (int t = threadIdx.x; t < b * npad; t += blockDim.x) {
            const int c = t / npad, i = t - c * npad;
            const int j = blk[s] * b + c;
            float* col = sb + (size_t)c * col_len;
            if (i > j) col[i] = 0.0f;
            if (i < nreal && j < nreal) Rsave[(size_t)j * nreal + i] = i > j ? 0.0f : col[i];
        }
    }
    __syncthreads();

    // ------------------------------------------------------------ sweeps --
    const float tol = 1.2e-7f * sqrtf((float)npad);
    const float tol2 = tol * tol;
    const int nv = npad / 4;                       // float4 vectors per column
    // one warp rotates columns x and y: c = x . y, then the plane rotation.
    // Every lane holds its share of both columns (at most NVL 16-byte
    // vectors of each) in registers from the first load to the store, so
    // the chain is one load, the dot product, the rotation's parameters and
    // one store.
    constexpr int NVL = C / 4;   // npad = 2 C b <= 32 C floats: 8 C vectors over 32 lanes
    // the rotation that zeroes x . y = c for squared norms a (x) and bb (y):
    // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) with zeta = (bb - a) / (2c), the
    // smaller root of t^2 + 2 zeta t - 1 = 0, written as 2c sign(d) / (|d| + sqrt(d^2 + 4c^2)),
    // d = bb - a: three dependent special-function operations instead of four
    // (the square root as h rsqrt(h), h > 0 since c != 0: the same few-ulp
    // accuracy as the rsqrt that gives cs).  The squared norms move by -t c
    // (x) and +t c (y).
    auto rot_params = [](float c, float a, float bb, float& cs, float& sn, float& tc) {
        const float d = bb - a;
        const float h = fmaf(d, d, 4.0f * c * c);
        const float t = __fdividef(d >= 0.0f ? 2.0f * c : -2.0f * c, fabsf(d) + h * rsqrtf(h));
        cs = rsqrtf(fmaf(t, t, 1.0f));
        sn = t * cs;
        tc = t * c;
    };
    auto rot4 = [](const float4& p, const float4& q, float cs, float sn, float4& o1, float4& o2) {
        const float4 r1 = make_float4(cs * p.x - sn * q.x, cs * p.y - sn * q.y, cs * p.z - sn * q.z, cs * p.w - sn * q.w);
        o2 = make_float4(sn * p.x + cs * q.x, sn * p.y + cs * q.y, sn * p.z + cs * q.z, sn * p.w + cs * q.w);
        o1 = r1;
    };
    // the largest (x . y)^2 / (|x|^2 |y|^2) this thread's warp met in the sweep
    float rmax2 = 0.0f;
    auto rotate_pair = [&](float* x, float* y, float* na, float* nb_, int ix, int iy) -> bool {
        float4* xw = reinterpret_cast<float4*>(x);
        float4* yw = reinterpret_cast<float4*>(y);
        const float a = *na, bb = *nb_;
        float4 px[NVL], qy[NVL];
        float c = 0.0f;
#pragma unroll
        for (int u = 0; u < NVL; ++u) {
            const int v = lane + 32 * u;
            if (v < nv) {
                px[u] = xw[v], qy[u] = yw[v];
            } else {
                px[u] = qy[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
            c += px[u].x * qy[u].x + px[u].y * qy[u].y + px[u].z * qy[u].z + px[u].w * qy[u].w;
        }
        c = warp_sum(c);
        if (ix >= nreal || iy >= nreal) return false;
        rmax2 = fmaxf(rmax2, __fdividef(c * c, a * bb));
        if (c == 0.0f || !(c * c > tol2 * (a * bb))) return false;
        float cs, sn, tc;
        rot_params(c, a, bb, cs, sn, tc);
#pragma unroll
        for (int u = 0; u < NVL; ++u) {
            const int v = lane + 32 * u;
            if (v < nv) {
                float4 o1, o2;
                rot4(px[u], qy[u], cs, sn, o1, o2);
                xw[v] = o1, yw[v] = o2;
            }
        }
        __syncwarp();
        if (lane == 0) {
            *na = a - tc;
            *nb_ = bb + tc;
        }
        return true;
    };
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        // column norms, recomputed every sweep
        for (int s = 0; s < 2; ++s) {
            float* sb = seat_buf(cur + s);
            for (int c = warp; c < b; c += JC_THREADS / 32) {
                const float4* xv = reinterpret_cast<const float4*>(sb + (size_t)c * col_len);
                float a = 0.0f;
                for (int v = lane; v < nv; v += 32) {
                    const float4 p = xv[v];
                    a += p.x * p.x + p.y * p.y + p.z * p.z + p.w * p.w;
                }
                a = warp_sum(a);
                if (lane == 0) nrm[(cur + s) * b + c] = a;
            }
        }
        if (threadIdx.x == 0) rot_flag = 0, rmax_bits = 0;
        rmax2 = 0.0f;
        __syncthreads();
        bool rotated = false;
        for (int br = 0; br < 2 * C - 1; ++br) {
            float* X = seat_buf(cur);
            float* Y = seat_buf(cur + 1);
            float* nX = nrm + cur * b;
            float* nY = nrm + (cur + 1) * b;
            const int* iX = idx + cur * b;
            const int* iY = idx + (cur + 1) * b;
            if (br == 0) {
                // pairs inside each block: round robin over b (+1 if odd) players
                const int bp = b + (b & 1);
                for (int r = 0; r < bp - 1; ++r) {
                    const int half = bp / 2;
                    if (warp < 2 * half) {
                        const int s = warp / half, k = warp - s * half;
                        const int u = (k == 0) ? bp - 1 : (r + k) % (bp - 1);
                        const int v = (k == 0) ? r : (r - k + bp - 1) % (bp - 1);
                        if (u < b && v < b) {
                            float* S = s ? Y : X;
                            float* nS = s ? nY : nX;
                            const int* iS = s ? iY : iX;
                            const int p = min(u, v), q = max(u, v);
                            rotated |= rotate_pair(S + (size_t)p * col_len, S + (size_t)q * col_len, nS + p, nS + q,
                                                   iS[p], iS[q]);
                        }
                    }
                    __syncthreads();
                }
            }
            // pairs between the two blocks: (X_i, Y_(i + r) mod b).  Warp i
            // keeps X_i and its norm in registers for the b
            // sub-rounds; only the Y columns pass through shared memory.
            {
                float4 px[NVL];
                float a = 0.0f;
                int ix = 0;
                if (warp < b) {
                    const float4* xw = reinterpret_cast<const float4*>(X + (size_t)warp * col_len);
#pragma unroll
                    for (int u = 0; u < NVL; ++u) {
                        const int v = lane + 32 * u;
                        px[u] = v < nv ? xw[v] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    }
                    a = nX[warp];
                    ix = iX[warp];
                }
                bool xdirty = false;
                for (int r = 0; r < b; ++r) {
                    if (warp < b) {
                        const int j = warp + r < b ? warp + r : warp + r - b;
                        float4* yw = reinterpret_cast<float4*>(Y + (size_t)j * col_len);
                        float4 qy[NVL];
                        const float bb = nY[j];
                        float c = 0.0f;
#pragma unroll
                        for (int u = 0; u < NVL; ++u) {
                            const int v = lane + 32 * u;
                            qy[u] = v < nv ? yw[v] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                            c += px[u].x * qy[u].x + px[u].y * qy[u].y + px[u].z * qy[u].z + px[u].w * qy[u].w;
                        }
                        c = warp_sum(c);
                        const bool real = ix < nreal && iY[j] < nreal;
                        if (real) rmax2 = fmaxf(rmax2, __fdividef(c * c, a * bb));
                        if (real && c != 0.0f && c * c > tol2 * (a * bb)) {
                            float cs, sn, tc;
                            rot_params(c, a, bb, cs, sn, tc);
#pragma unroll
                            for (int u = 0; u < NVL; ++u) {
                                const int v = lane + 32 * u;
                                float4 o;
                                rot4(px[u], qy[u], cs, sn, px[u], o);
                                if (v < nv) yw[v] = o;
                            }
                            a -= tc;
                            if (lane == 0) nY[j] = bb + tc;
                            rotated = xdirty = true;
                        }
                    }
                    __syncthreads();
                }
                if (warp < b && xdirty) {
                    float4* xw = reinterpret_cast<float4*>(X + (size_t)warp * col_len);
#pragma unroll
                    for (int u = 0; u < NVL; ++u) {
                        const int v = lane + 32 * u;
                        if (v < nv) xw[v] = px[u];
                    }
                    if (lane == 0) nX[warp] = a;
                }
                __syncthreads();
            }
            // move the blocks to the next seats (seat 0 stays, seat k -> k + 1, 2C - 1 -> 1)
            cluster.sync();
            const int nxt = cur ^ 2;
            for (int s = 0; s < 2; ++s) {
                const int seat = s == 0 ? rank : 2 * C - 1 - rank;
                int src_seat = seat == 0 ? 0 : (seat == 1 ? 2 * C - 1 : seat - 1);
                const int src_rank = src_seat < C ? src_seat : 2 * C - 1 - src_seat;
                const int src_s = src_seat < C ? 0 : 1;
                const float* sb = cluster.map_shared_rank(seat_buf(cur + src_s), src_rank);
                const float* sn = cluster.map_shared_rank(nrm + (cur + src_s) * b, src_rank);
                const int* si = cluster.map_shared_rank(idx + (cur + src_s) * b, src_rank);
                float4* dst = reinterpret_cast<float4*>(seat_buf(nxt + s));
                const float4* src = reinterpret_cast<const float4*>(sb);
                // four remote loads in flight per thread before the stores
                const int nvec = slot_len / 4;
                for (int v0 = threadIdx.x; v0 < nvec; v0 += 4 * JC_THREADS) {
                    float4 t4[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int v = v0 + u * JC_THREADS;
                        if (v < nvec) t4[u] = src[v];
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int v = v0 + u * JC_THREADS;
                        if (v < nvec) dst[v] = t4[u];
                    }
                }
                for (int c = threadIdx.x; c < b; c += blockDim.x) {
                    nrm[(nxt + s) * b + c] = sn[c];
                    idx[(nxt + s) * b + c] = si[c];
                }
            }
            // a block barrier suffices here: the buffers just read in other
            // CTAs (their current seats) are next written by the copy of the
            // following move, after its cluster barrier, which every CTA
            // reaches only once this copy is done
            __syncthreads();
            cur = nxt;
        }
        // cluster-wide vote: did any pair rotate in this sweep?
        if (rotated) atomicOr(&rot_flag, 1);
        // non-negative floats order as their bit patterns
        if (lane == 0) atomicMax(&rmax_bits, __float_as_int(rmax2));
        cluster.sync();
        int any = 0;
        float cmax2 = 0.0f;
#pragma unroll 1
        for (int r = 0; r < C; ++r) {
            any |= *cluster.map_shared_rank(&rot_flag, r);
            cmax2 = fmaxf(cmax2, __int_as_float(*cluster.map_shared_rank(&rmax_bits, r)));
        }
        cluster.sync();
        if (!any || cmax2 < stop2) {
            ++sweep;
            break;
        }
    }
    // the columns of R V out, at the index each column started from
    for (int s = 0; s < 2; ++s) {
        const float* sb = seat_buf(cur + s);
        for (int t = threadIdx.x; t < b * nreal; t += blockDim.x) {
            const int c = t / nreal, i = t - c * nreal;
            const int j = idx[(cur + s) * b + c];
            if (j < nreal) V[(size_t)i * ldv + j] = sb[(size_t)c * col_len + i];
        }
    }
    if (rank == 0 && threadIdx.x == 0) {
        *sweeps_out = sweep;
        *status_out = 0;
    }
}

// V := R^{-1} V column by column, then each column scaled to unit length:
// R upper triangular (nreal x nreal, column-major, ld nreal, as the cluster
// kernel saved it), V row-major with ld ldv.  One CTA per column; rows in
// blocks of 32 from the bottom: one warp solves the block's triangle (its
// 32 x 32 part of R in registers, the solution broadcast by shuffles), then
// every thread removes the block from the rows above.  Nothing is done when
// *status != 0 (the cluster kernel's Cholesky failed and the two-sided
// kernel writes V instead).
__global__ void __launch_bounds__(256) jc_backsolve_kernel(const float* __restrict__ R, float* __restrict__ V,
                                                           int ldv, int nreal, const int* __restrict__ status) {
    if (*status != 0) return;
    extern __shared__ float y[];   // nreal
    __shared__ float red[8];
    const int j = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < nreal; i += blockDim.x) y[i] = V[(size_t)i * ldv + j];
    __syncthreads();
    for (int i1 = nreal; i1 > 0; i1 -= 32) {
        const int i0 = i1 > 32 ? i1 - 32 : 0, m = i1 - i0;
        if (warp == 0) {
            // lane l: row i0 + l; rt[t] = R(i0 + l, i0 + t) for l <= t < m
            float rt[32];
#pragma unroll
            for (int t = 0; t < 32; ++t)
                rt[t] = (t < m && lane <= t) ? R[(size_t)(i0 + t) * nreal + i0 + lane] : 0.0f;
            float yl = lane < m ? y[i0 + lane] : 0.0f;
#pragma unroll
            for (int t = 31; t >= 0; --t) {
                if (t < m) {
                    const float xt = __shfl_sync(0xffffffffu, lane == t ? yl / rt[t] : 0.0f, t);
                    if (lane == t) yl = xt;
                    else if (lane < t) yl = fmaf(-rt[t], xt, yl);
                }
            }
            if (lane < m) y[i0 + lane] = yl;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < i0; k += blockDim.x) {
            float acc = 0.0f;
            for (int t = 0; t < m; ++t) acc = fmaf(R[(size_t)(i0 + t) * nreal + k], y[i0 + t], acc);
            y[k] -= acc;
        }
        __syncthreads();
    }
    float ss = 0.0f;
    for (int i = threadIdx.x; i < nreal; i += blockDim.x) ss = fmaf(y[i], y[i], ss);
    ss = warp_sum(ss);
    if (lane == 0) red[warp] = ss;
    __syncthreads();
    float tot = 0.0f;
#pragma unroll
    for (int w = 0; w < 8; ++w) tot += red[w];
    const float sc = tot > 0.0f ? rsqrtf(tot) : 0.0f;
    for (int i = threadIdx.x; i < nreal; i += blockDim.x) V[(size_t)i * ldv + j] = y[i] * sc;
}

template <int C>
int launch_jc(nys_ctx* ctx, const double* G, int ell, int b, int max_sweeps, float* V, int ldv, float* Rsave,
              int* sweeps, int* status) {
    const int npad = 2 * C * b;
    const size_t smem = (size_t)4 * b * npad * sizeof(float) + (size_t)4 * b * (sizeof(float) + sizeof(int)) + 64;
    if (smem > 220 * 1024) return NYS_EINVAL;
    auto k = jacobi_cluster_kernel<C>;
    if (C > 8) NYS_CK(ctx, cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    if (int st = smem_optin(ctx, (const void*)k, smem)) return st;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(JC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k, &cfg) != cudaSuccess || clusters < 1) {
        cudaGetLastError();
        return NYS_EINVAL;
    }
    // stop after a sweep whose largest |x . y| / (|x| |y|) was below 1e-3: its
    // rotations leave off-diagonal terms of the order of its square, at the
    // float32 floor of the test (quadratic convergence), so the sweep that
    // would only confirm it is skipped
    NYS_CK(ctx, cudaLaunchKernelEx(&cfg, k, G, ell, b, max_sweeps, V, ldv, Rsave, 1e-6f, sweeps, status));
    ++ctx->launches;
    jc_backsolve_kernel<<<ell, 256, (size_t)ell * sizeof(float), ctx->stream>>>(Rsave, V, ldv, ell, status);
    NYS_LAUNCH_CK(ctx);
    return NYS_OK;
}

}  // namespace

// V (row-major, ld = ldv, float32) = eigenvectors of the symmetric ell x ell
// float64 matrix G by the cluster kernel and the back substitution above;
// Rsave: ell * ell floats of device workspace.  NYS_EINVAL (nothing
// launched) when ell is outside [64, 448] or the cluster cannot be placed.
// *status = 1 on the device if the float32 Cholesky of G fails (V is then
// not written).
int jacobi_cluster(nys_ctx* ctx, const double* G, int ell, int max_sweeps, float* V, int ldv, float* Rsave,
                   int* sweeps, int* status) {
    if (ell < 64 || ell > 448) return NYS_EINVAL;
    if (ell <= 256) return launch_jc<8>(ctx, G, ell, (ell + 15) / 16, max_sweeps, V, ldv, Rsave, sweeps, status);
    return launch_jc<16>(ctx, G, ell, (ell + 31) / 32, max_sweeps, V, ldv, Rsave, sweeps, status);
}

}  // namespace nys
