// Parallel-beam ray transform A and its exact transpose A^T (Sec. IV-C, the CT
// forward model), discretised with Joseph's method (P. M. Joseph, "An improved
// algorithm for reprojecting rays through pixel images", IEEE TMI 1982).
//
// Geometry: pixel (i, j) sits at x = j - c2, y = i - c1 (c = (n-1)/2); ray
// (theta_k, t_m) is the line x cos + y sin = t with theta_k = k span / n_angles
// and t_m = m - (n_bins - 1)/2.  A "row-step" angle (|cos| + 1e-9 >= |sin|)
// samples the ray once per image row i at column position
//     u(i, m) = c2 + t_m / cos - (i - c1) tan = Q_m + R_i
// with linear interpolation between columns floor(u) and floor(u) + 1 and
// weight 1/|cos|; a "column-step" angle swaps the roles of rows and columns
// (Q_m = c1 + t_m / sin, R_j = -(j - c2) cot, weight 1/|sin|).  Samples that
// fall outside the image contribute zero.
//
// Precision: Q_m and R_l are split on the host, in float64, into an integer
// part and a fraction in [0, 1).  The device adds the two fractions (error at
// most one float ulp of a number below 2), so interpolation weights carry an
// absolute error near 1e-7 instead of the ~3e-5 that a float position near 500
// would carry.  The forward (ray-driven) and the adjoint (pixel-driven gather)
// evaluate the SAME float expressions for every (ray, line) pair, so the
// adjoint is the exact transpose of the forward up to summation order, with
// no atomics.
//
// Forward: one CTA per (angle, group of IB images), each warp 96 consecutive
// bins (three per lane), stepping along the lines of the angle that the
// warp's rays cross inside the image.  The image is read "line-major":
// row-step angles read the row-major image, column-step angles a transposed
// copy (made once per batch chunk), so consecutive bins of a warp read
// consecutive addresses for both kinds of angle.  The per-line table entries
// are staged in shared memory and shared by the three bins and the IB images.
// Adjoint: one CTA per (16 x 16 pixel tile, group of IB images).  Angles are
// taken AK at a time: for each, the window of bins that can reach the tile
// (from the four tile corners) is staged in shared memory with its tables and
// sinogram values, so the per-pixel candidate tests read shared memory only;
// candidates outside the window (none for |slope| <= 1, kept for safety) fall
// back to global loads.
#include "internal.cuh"

#include <cmath>
#include <type_traits>

namespace nys {
namespace {

template <class TC>
struct RTab {
    const int* qi;     // [n_angles][n_bins]
    const TC* qf;      // [n_angles][n_bins]
    const int* ri;     // [n_angles][nl_max]
    const TC* rf;      // [n_angles][nl_max]
    const TC* wt;      // [n_angles] 1/|cos| or 1/|sin|
    const TC* slope;   // [n_angles] dm/du = cos (row-step) or sin (column-step)
    const TC* oth;     // [n_angles] sin (row-step) or cos (column-step): dm*/dl
    const int* rowstep;// [n_angles]
    int nl_max;
};

template <class TC>
__device__ __forceinline__ void sample_pos(int qi, TC qf, int ri, TC rf, int& lo, TC& w) {
    TC f = qf + rf;
    const int carry = f >= TC(1) ? 1 : 0;
    f -= (TC)carry;
    lo = qi + ri + carry;
    w = f;
}

// xr (optional) / xT: line-major copies of `batch` images in the compute type;
// xT[b][j][i] = x[b][i][j]
template <class TI, class TC>
__global__ void radon_prep_kernel(const TI* __restrict__ x, TC* __restrict__ xr, TC* __restrict__ xT, int n1, int n2) {
    pdl_enter();
    __shared__ TC tile[32][33];
    const int b = blockIdx.z;
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const TI* xb = x + (size_t)b * n1 * n2;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        TC v = TC(0);
        if (i < n1 && j < n2) {
            v = (TC)ldf(xb + (size_t)i * n2 + j);
            if (xr) xr[(size_t)b * n1 * n2 + (size_t)i * n2 + j] = v;
        }
        tile[r][threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r, i = i0 + threadIdx.x;
        if (i < n1 && j < n2) xT[(size_t)b * n1 * n2 + (size_t)j * n1 + i] = tile[threadIdx.x][r];
    }
}

// forward: one CTA per (angle, IB images); warps over bins, three per lane
template <class TC, class TO, int IB>
__global__ void __launch_bounds__(256) radon_fwd2_kernel(const TC* __restrict__ xr, const TC* __restrict__ xT,
                                                         TO* __restrict__ y, int n1, int n2, int n_angles,
                                                         int n_bins, int batch, RTab<TC> tab) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int k = blockIdx.x;
    const int b0 = blockIdx.y * IB;
    const int rs = tab.rowstep[k];
    const int nl = rs ? n1 : n2;       // lines (rows for row-step)
    const int na = rs ? n2 : n1;       // positions along a line
    int* s_ri = reinterpret_cast<int*>(smem_raw);
    TC* s_rf = reinterpret_cast<TC*>(s_ri + ((nl + 3) & ~3));
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
        s_ri[l] = tab.ri[(size_t)k * tab.nl_max + l];
        s_rf[l] = tab.rf[(size_t)k * tab.nl_max + l];
    }
    __syncthreads();
    const size_t N = (size_t)n1 * n2;
    const TC* src = (rs ? xr : xT) + (size_t)b0 * N;
    const TC wt = tab.wt[k];
    // a warp takes 96 consecutive bins (three groups of 32, one bin of each
    // per lane: the loads of a group stay coalesced)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    // u(m, l) = Q_m + R_l with R_l = -(l - c_line) t, t = oth / den: the
    // lines where a sample of the warp's bins can land in [-1, na) form one
    // interval (Q is monotone in m), taken with two lines of margin; outside
    // it every sample is out of range and adds exactly zero
    const TC tl = tab.oth[k] / tab.slope[k];
    const TC c_line = TC(0.5) * (TC)((rs ? n1 : n2) - 1);
    for (int mb = warp * 96 + lane; mb - lane < n_bins; mb += nw * 96) {
        const int mf = mb - lane, ml = min(mf + 95, n_bins - 1);
        const TC Qa = (TC)tab.qi[(size_t)k * n_bins + mf] + tab.qf[(size_t)k * n_bins + mf];
        const TC Qb = (TC)tab.qi[(size_t)k * n_bins + ml] + tab.qf[(size_t)k * n_bins + ml];
        const TC Qmin = fmin(Qa, Qb), Qmax = fmax(Qa, Qb);
        int l_beg = 0, l_end = nl;
        if (fabs(tl) > TC(1e-6)) {
            // -1 <= Q - (l - c_line) t < na
            const TC e1 = c_line + (Qmin - (TC)na) / tl, e2 = c_line + (Qmax + TC(1)) / tl;
            l_beg = max(0, (int)floor(fmin(e1, e2)) - 2);
            l_end = min(nl, (int)ceil(fmax(e1, e2)) + 3);
        } else if (Qmax < TC(-3) || Qmin > (TC)(na + 2)) {
            l_end = 0;
        }
        int qi[3];
        TC qf[3];
        bool ok[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int m = mb + c * 32;
            ok[c] = m < n_bins;
            // a bin past the last one gets a position far below the line, so
            // the range tests below reject it without a separate flag
            qi[c] = ok[c] ? tab.qi[(size_t)k * n_bins + m] : -(1 << 28);
            qf[c] = ok[c] ? tab.qf[(size_t)k * n_bins + m] : TC(0);
        }
        TC acc[3][IB];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 0; q < IB; ++q) acc[c][q] = TC(0);
#pragma unroll 4
        for (int l = l_beg; l < l_end; ++l) {
            const int ri = s_ri[l];
            const TC rf = s_rf[l];
            const TC* line = src + (size_t)l * na;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                int lo;
                TC w;
                sample_pos<TC>(qi[c], qf[c], ri, rf, lo, w);
                const bool in0 = (unsigned)lo < (unsigned)na, in1 = (unsigned)(lo + 1) < (unsigned)na;
#pragma unroll
                for (int q = 0; q < IB; ++q) {
                    const TC* lq = line + (size_t)q * N;
                    const bool live = b0 + q < batch;
                    const TC v0 = (in0 && live) ? lq[lo] : TC(0);
                    const TC v1 = (in1 && live) ? lq[lo + 1] : TC(0);
                    acc[c][q] = fma(TC(1) - w, v0, acc[c][q]);
                    acc[c][q] = fma(w, v1, acc[c][q]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int m = mb + c * 32;
            if (!ok[c]) continue;
#pragma unroll
            for (int q = 0; q < IB; ++q)
                if (b0 + q < batch) stf(y + ((size_t)(b0 + q) * n_angles + k) * n_bins + m, wt * acc[c][q]);
        }
    }
}

// adjoint, line-scatter form: one CTA per (16 x 16 pixel tile, IB images),
// AK angles per round.  The 256 threads are (angle a, segment g, line r) with
// r over the tile's 16 lines (tile rows for a row-step angle, tile columns for
// a column-step one) and AK x S = 16 (S = 16 / AK segments of the line's
// bins).  A thread walks its bins in increasing order, evaluates the
// forward's sample position with the same float expressions (sample_pos) and
// adds (1 - f) s[m] at position lo and f s[m] at lo + 1 into its own row of a
// shared buffer: no other thread writes that row, so there are no races and
// the order of the sums is fixed.  After a barrier each pixel adds, angle by
// angle, the S segment entries of its position and then the weighted angle
// term -- the exact transpose of the forward, up to summation order.  The
// global loads of the next round (staged bins, sinogram values, the line's
// table entry) are issued into registers before the current round's scatter.
constexpr int ATS = 16;     // tile side
// staged bins per angle: the bins reaching a line of the tile start at most
// 4 + 1 bins above the window start and span 17 |slope| + 15 |oth| + 2 <= 25
// more (|slope|, |oth| <= 1 and 17^2 + 15^2 < 23^2), so 32 cover them all
constexpr int AWIN = 32;
constexpr int AWP = AWIN + 16;   // sinogram row pitch: the two angles of a warp 16 banks apart

template <class TC>
struct QS {   // one staged bin: integer and fractional part of Q_m
    int qi;
    TC qf;
};

template <class TI, class TO, class TC, int IB, int AK>
__global__ void __launch_bounds__(256, IB == 1 ? 6 : 2)
    radon_adj3_kernel(const TI* __restrict__ s, TO* __restrict__ x, int n1, int n2, int n_angles, int n_bins,
                      int batch, RTab<TC> tab, TC c1, TC c2, TC cb) {
    pdl_enter();
    constexpr int S = ATS / AK;            // segments per line
    constexpr int BP = ATS + 1;            // buffer row pitch (odd: spreads the banks)
    constexpr int U = (AK * AWIN + 255) / 256;   // staged entries per thread
    static_assert(AK * S == ATS, "AK divides the tile side");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // [buf: AK S x IB x 16 x BP][sqs: AK x AWIN][ss: AK x IB x AWP][slope, oth, wt: n_angles]
    // [rowstep: n_angles][mlo: AK]
    TC* buf = reinterpret_cast<TC*>(smem_raw);
    QS<TC>* sqs = reinterpret_cast<QS<TC>*>(buf + AK * S * IB * ATS * BP);
    TC* ss = reinterpret_cast<TC*>(sqs + AK * AWIN);
    TC* g_slope = ss + AK * IB * AWP;
    TC* g_oth = g_slope + n_angles;
    TC* g_wt = g_oth + n_angles;
    int* g_rs = reinterpret_cast<int*>(g_wt + n_angles);
    int* s_mlo = g_rs + n_angles;
    const int i0 = blockIdx.y * ATS, j0 = blockIdx.x * ATS;
    const int b0 = blockIdx.z * IB;
    const int ti = threadIdx.x / ATS, tj = threadIdx.x % ATS;
    const int i = i0 + ti, j = j0 + tj;
    const bool valid = i < n1 && j < n2;
    // scatter role: line r of angle a_me, segment g_me
    const int r = threadIdx.x % ATS, a_me = (threadIdx.x / ATS) / S, g_me = (threadIdx.x / ATS) % S;
    const size_t M = (size_t)n_angles * n_bins;
    for (int k = threadIdx.x; k < n_angles; k += blockDim.x) {
        g_rs[k] = tab.rowstep[k];
        g_slope[k] = tab.slope[k];
        g_oth[k] = tab.oth[k];
        g_wt[k] = tab.wt[k];
    }
    __syncthreads();
    // first staged bin of angle k for this tile: m* = cb + slope (p - cpos) + oth (l - cline)
    // is affine in (p, l), so its minimum over the tile (positions one beyond
    // each side included) is at a corner; four bins of margin cover the float
    // rounding of the split tables
    auto window = [&](int k) -> int {
        const int rs = g_rs[k];
        const TC sl = g_slope[k], ot = g_oth[k];
        const TC pa = (TC)(rs ? j0 : i0) - (rs ? c2 : c1);
        const TC la = (TC)(rs ? i0 : j0) - (rs ? c1 : c2);
        const TC mp = fmin(sl * (pa - TC(1)), sl * (pa + TC(ATS)));
        const TC ml = fmin(ot * la, ot * (la + TC(ATS - 1)));
        return (int)floor(cb + mp + ml) - 4;
    };
    // next round's loads, held in registers through the current round
    int pf_qi[U];
    TC pf_qf[U];
    TC pf_s[U][IB];
    int pf_ri = 0;
    TC pf_rf = TC(0);
    auto prefetch = [&](int k0) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = threadIdx.x + 256 * u;
            const int a = e / AWIN, w = e % AWIN;
            const int k = k0 + a;
            bool ok = e < AK * AWIN && k < n_angles;
            const int m = ok ? window(k) + w : 0;
            ok = ok && m >= 0 && m < n_bins;
            pf_qi[u] = ok ? tab.qi[(size_t)k * n_bins + m] : 0;
            pf_qf[u] = ok ? tab.qf[(size_t)k * n_bins + m] : TC(0);
#pragma unroll
            for (int q = 0; q < IB; ++q)
                pf_s[u][q] = (ok && b0 + q < batch) ? (TC)ldf(s + (size_t)(b0 + q) * M + (size_t)k * n_bins + m) : TC(0);
        }
        const int k = k0 + a_me;
        pf_ri = 0;
        pf_rf = TC(0);
        if (k < n_angles) {
            const int rs = g_rs[k];
            const int l = (rs ? i0 : j0) + r;
            if (l < (rs ? n1 : n2)) {
                pf_ri = tab.ri[(size_t)k * tab.nl_max + l];
                pf_rf = tab.rf[(size_t)k * tab.nl_max + l];
            }
        }
    };
    TC acc[IB];
#pragma unroll
    for (int q = 0; q < IB; ++q) acc[q] = TC(0);
    prefetch(0);
    for (int k0 = 0; k0 < n_angles; k0 += AK) {
        __syncthreads();   // the previous round's buffers and tables are consumed
        if (threadIdx.x < AK) s_mlo[threadIdx.x] = (k0 + threadIdx.x < n_angles) ? window(k0 + threadIdx.x) : 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = threadIdx.x + 256 * u;
            if (e < AK * AWIN) {
                const int a = e / AWIN, w = e % AWIN;
                sqs[e] = QS<TC>{pf_qi[u], pf_qf[u]};
#pragma unroll
                for (int q = 0; q < IB; ++q) ss[(a * IB + q) * AWP + w] = pf_s[u][q];
            }
        }
        const int ri = pf_ri;
        const TC rf = pf_rf;
        // zero this thread's buffer rows (only it writes them)
        TC* row = buf + (size_t)((a_me * S + g_me) * IB) * ATS * BP;
        const int k_me = k0 + a_me;
        const int rs = k_me < n_angles ? g_rs[k_me] : 1;
        // row-step: line r is tile row r, position c is column c -> [r][c];
        // column-step: line r is tile column r, position c is row c -> [c][r]
        const int ls = rs ? BP : 1, ps = rs ? 1 : BP;
#pragma unroll
        for (int q = 0; q < IB; ++q)
            for (int c = 0; c < ATS; ++c) row[q * ATS * BP + r * ls + c * ps] = TC(0);
        __syncthreads();
        if (k0 + AK < n_angles) prefetch(k0 + AK);
        const int l = (rs ? i0 : j0) + r;              // line index in the image
        if (k_me < n_angles && l < (rs ? n1 : n2)) {
            const int p0 = rs ? j0 : i0;               // first position of the tile on the line
            const TC cpos = rs ? c2 : c1;
            const TC sl = g_slope[k_me];
            // bins whose sample lands in positions p0 - 1 .. p0 + 15 (u in
            // [p0 - 1, p0 + 16)), from the inverse m*(p) with one bin of
            // margin; they lie inside the staged window (see AWIN)
            const TC base = cb - sl * (cpos + ((TC)ri + rf));
            const TC ma = base + sl * (TC)(p0 - 1), mb = base + sl * (TC)(p0 + ATS);
            const int wlo = s_mlo[a_me];
            const int mlo = max(max(0, wlo), (int)floor(fmin(ma, mb)) - 1);
            const int mhi = min(min(n_bins, wlo + AWIN) - 1, (int)ceil(fmax(ma, mb)) + 1);
            const int len = mhi - mlo + 1;
            if (len > 0) {
                const int w_beg = mlo - wlo + (g_me * len) / S, w_end = mlo - wlo + ((g_me + 1) * len) / S;
                const QS<TC>* qa = sqs + a_me * AWIN;
                const TC* sa = ss + a_me * IB * AWP;
                TC* rl = row + r * ls;
                if constexpr (IB == 1) {
                    // one image: read-modify-write of the buffer row
                    for (int w = w_beg; w < w_end; ++w) {
                        const QS<TC> e = qa[w];
                        int lo;
                        TC f;
                        sample_pos<TC>(e.qi, e.qf, ri, rf, lo, f);
                        const int c = lo - p0;
                        if (c < -1 || c >= ATS) continue;
                        const TC sv = sa[w];
                        if (c >= 0) rl[c * ps] = fma(TC(1) - f, sv, rl[c * ps]);
                        if (c + 1 < ATS) rl[(c + 1) * ps] = fma(f, sv, rl[(c + 1) * ps]);
                    }
                } else {
                    // Several images: two positions are summed in registers and
                    // each is written out once (fewer shared-memory accesses per
                    // bin; measured faster for 4 images per CTA, slower for one).
                    // lo is monotone in m, so a position's (at most two, three on
                    // a rounding tie) contributions come from consecutive bins,
                    // and a slot is complete as soon as a bin no longer touches
                    // it.  The sums run in bin order, as the read-modify-write.
                    int cA = -1000, cB = -1000;
                    TC vA[IB], vB[IB];
#pragma unroll
                    for (int q = 0; q < IB; ++q) vA[q] = vB[q] = TC(0);
                    auto flush = [&](int c, const TC* v) {
                        if (c >= 0 && c < ATS) {
#pragma unroll
                            for (int q = 0; q < IB; ++q) rl[q * ATS * BP + c * ps] = v[q];
                        }
                    };
                    for (int w = w_beg; w < w_end; ++w) {
                        const QS<TC> e = qa[w];
                        int lo;
                        TC f;
                        sample_pos<TC>(e.qi, e.qf, ri, rf, lo, f);
                        const int c = lo - p0;
                        if (c < -1 || c >= ATS) continue;
                        TC sv[IB];
#pragma unroll
                        for (int q = 0; q < IB; ++q) sv[q] = sa[q * AWP + w];
#pragma unroll
                        for (int t = 0; t < 2; ++t) {          // position c (weight 1 - f), then c + 1 (f)
                            const int ct = c + t;
                            const TC wgt = t ? f : TC(1) - f;
                            if (ct == cA) {
#pragma unroll
                                for (int q = 0; q < IB; ++q) vA[q] = fma(wgt, sv[q], vA[q]);
                            } else if (ct == cB) {
#pragma unroll
                                for (int q = 0; q < IB; ++q) vB[q] = fma(wgt, sv[q], vB[q]);
                            } else if (cA != c && cA != c + 1) {   // slot A is complete
                                flush(cA, vA);
                                cA = ct;
#pragma unroll
                                for (int q = 0; q < IB; ++q) vA[q] = fma(wgt, sv[q], TC(0));
                            } else {                               // slot B is
                                flush(cB, vB);
                                cB = ct;
#pragma unroll
                                for (int q = 0; q < IB; ++q) vB[q] = fma(wgt, sv[q], TC(0));
                            }
                        }
                    }
                    flush(cA, vA);
                    flush(cB, vB);
                }
            }
        }
        __syncthreads();
        if (!valid) continue;
        const int na = min(AK, n_angles - k0);
        for (int a = 0; a < na; ++a) {
#pragma unroll
            for (int q = 0; q < IB; ++q) {
                TC part = buf[(size_t)((a * S) * IB + q) * ATS * BP + ti * BP + tj];
#pragma unroll
                for (int g = 1; g < S; ++g) part += buf[(size_t)((a * S + g) * IB + q) * ATS * BP + ti * BP + tj];
                acc[q] = fma(g_wt[k0 + a], part, acc[q]);
            }
        }
    }
    if (!valid) return;
#pragma unroll
    for (int q = 0; q < IB; ++q)
        if (b0 + q < batch) stf(x + ((size_t)(b0 + q) * n1 + i) * n2 + j, acc[q]);
}

template <class TC>
void split(double v, int& I, TC& F) {
    double fl = std::floor(v);
    double fr = v - fl;
    TC f = (TC)fr;
    if (f >= TC(1)) {
        f = TC(0);
        fl += 1.0;
    }
    I = (int)fl;
    F = f;
}

template <class TC>
int build_tables(nys_op* op) {
    const int A = op->n_angles, B = op->n_bins, n1 = op->n1, n2 = op->n2;
    const int nl_max = std::max(n1, n2);
    const double c1 = (n1 - 1) / 2.0, c2 = (n2 - 1) / 2.0, cb = (B - 1) / 2.0;
    std::vector<int> qi((size_t)A * B), ri((size_t)A * nl_max, 0), rowstep(A);
    std::vector<TC> qf((size_t)A * B), rf((size_t)A * nl_max, TC(0)), wt(A), slope(A), othv(A);
    for (int k = 0; k < A; ++k) {
        const double th = k * (op->span / A);
        const double cs = std::cos(th), sn = std::sin(th);
        const bool rs = std::fabs(cs) + 1e-9 >= std::fabs(sn);
        rowstep[k] = rs;
        const double c_line = rs ? c1 : c2;   // centre of the line index
        const double c_pos = rs ? c2 : c1;
        const double den = rs ? cs : sn;      // u = c_pos + t/den - (l - c_line) * other/den
        const double oth = rs ? sn : cs;
        wt[k] = (TC)(1.0 / std::fabs(den));
        slope[k] = (TC)den;
        othv[k] = (TC)oth;
        for (int m = 0; m < B; ++m) split<TC>(c_pos + (m - cb) / den, qi[(size_t)k * B + m], qf[(size_t)k * B + m]);
        const int nl = rs ? n1 : n2;
        for (int l = 0; l < nl; ++l)
            split<TC>(-(l - c_line) * oth / den, ri[(size_t)k * nl_max + l], rf[(size_t)k * nl_max + l]);
    }
    size_t off = 0;
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    const size_t sz_qi = al(qi.size() * 4), sz_qf = al(qf.size() * sizeof(TC)), sz_ri = al(ri.size() * 4),
                 sz_rf = al(rf.size() * sizeof(TC)), sz_a = al(A * sizeof(TC)), sz_rs = al(A * 4);
    const size_t total = sz_qi + sz_qf + sz_ri + sz_rf + 3 * sz_a + sz_rs;
    NYS_CK(op->ctx, cudaMalloc(&op->rtab, total));
    char* base = (char*)op->rtab;
    auto put = [&](const void* src, size_t n, size_t sz) {
        cudaError_t e = cudaMemcpy(base + off, src, n, cudaMemcpyHostToDevice);
        off += sz;
        return e;
    };
    NYS_CK(op->ctx, put(qi.data(), qi.size() * 4, sz_qi));
    NYS_CK(op->ctx, put(qf.data(), qf.size() * sizeof(TC), sz_qf));
    NYS_CK(op->ctx, put(ri.data(), ri.size() * 4, sz_ri));
    NYS_CK(op->ctx, put(rf.data(), rf.size() * sizeof(TC), sz_rf));
    NYS_CK(op->ctx, put(wt.data(), A * sizeof(TC), sz_a));
    NYS_CK(op->ctx, put(slope.data(), A * sizeof(TC), sz_a));
    NYS_CK(op->ctx, put(othv.data(), A * sizeof(TC), sz_a));
    NYS_CK(op->ctx, put(rowstep.data(), A * 4, sz_rs));
    return NYS_OK;
}

template <class TC>
RTab<TC> tables(const nys_op* op) {
    const int A = op->n_angles, B = op->n_bins;
    const int nl_max = std::max(op->n1, op->n2);
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    const char* base = (const char*)op->rtab;
    RTab<TC> t;
    size_t off = 0;
    t.qi = (const int*)(base + off);
    off += al((size_t)A * B * 4);
    t.qf = (const TC*)(base + off);
    off += al((size_t)A * B * sizeof(TC));
    t.ri = (const int*)(base + off);
    off += al((size_t)A * nl_max * 4);
    t.rf = (const TC*)(base + off);
    off += al((size_t)A * nl_max * sizeof(TC));
    t.wt = (const TC*)(base + off);
    off += al(A * sizeof(TC));
    t.slope = (const TC*)(base + off);
    off += al(A * sizeof(TC));
    t.oth = (const TC*)(base + off);
    off += al(A * sizeof(TC));
    t.rowstep = (const int*)(base + off);
    t.nl_max = nl_max;
    return t;
}

template <class TI, class TO, class TC>
int radon_fwd(nys_op* op, const void* x, void* y, int batch) {
    const int nl_max = std::max(op->n1, op->n2);
    const size_t sm = ((nl_max + 3) & ~3) * 4 + nl_max * sizeof(TC);
    const size_t N = (size_t)op->N;
    cudaStream_t st = op->ctx->stream;
    TC* xT = (TC*)op->lines;
    TC* xr = xT + (size_t)op->chunk * N;
    for (int b0 = 0; b0 < batch; b0 += op->chunk) {
        const int nb = std::min(op->chunk, batch - b0);
        const TI* xb = (const TI*)x + (size_t)b0 * N;
        // the row-major source is x itself when it already has the compute type
        const bool same = std::is_same<TI, TC>::value;
        NYS_CK(op->ctx, launch_pdl(radon_prep_kernel<TI, TC>, dim3((op->n2 + 31) / 32, (op->n1 + 31) / 32, nb),
                                   dim3(32, 8), 0, st, xb, same ? nullptr : xr, xT, op->n1, op->n2));
        NYS_LAUNCH_CK(op->ctx);
        const TC* src_r = same ? (const TC*)xb : xr;
        TO* yb = (TO*)y + (size_t)b0 * op->M;
        if (nb >= 4) {
            const int full = nb / 4 * 4;
            NYS_CK(op->ctx, launch_pdl(radon_fwd2_kernel<TC, TO, 4>, dim3(op->n_angles, full / 4), 256, sm, st, src_r,
                                       (const TC*)xT, yb, op->n1, op->n2, op->n_angles, op->n_bins, full,
                                       tables<TC>(op)));
            NYS_LAUNCH_CK(op->ctx);
            if (full < nb) {
                NYS_CK(op->ctx, launch_pdl(radon_fwd2_kernel<TC, TO, 1>, dim3(op->n_angles, nb - full), 256, sm, st,
                                           src_r + (size_t)full * N, (const TC*)(xT + (size_t)full * N),
                                           yb + (size_t)full * op->M, op->n1, op->n2, op->n_angles, op->n_bins,
                                           nb - full, tables<TC>(op)));
                NYS_LAUNCH_CK(op->ctx);
            }
        } else {
            NYS_CK(op->ctx, launch_pdl(radon_fwd2_kernel<TC, TO, 1>, dim3(op->n_angles, nb), 256, sm, st, src_r,
                                       (const TC*)xT, yb, op->n1, op->n2, op->n_angles, op->n_bins, nb,
                                       tables<TC>(op)));
            NYS_LAUNCH_CK(op->ctx);
        }
    }
    return NYS_OK;
}

template <class TC, int IB, int AK>
size_t adj3_smem(int n_angles) {
    constexpr int S = ATS / AK;
    return sizeof(TC) * ((size_t)AK * S * IB * ATS * (ATS + 1) + (size_t)AK * IB * AWP + 3 * (size_t)n_angles) +
           sizeof(QS<TC>) * (size_t)AK * AWIN + sizeof(int) * ((size_t)n_angles + AK);
}

template <class TI, class TO, class TC, int IB, int AK>
void radon_adj_launch(nys_op* op, const TI* s, TO* x, int nb) {
    dim3 grid((op->n2 + ATS - 1) / ATS, (op->n1 + ATS - 1) / ATS, (nb + IB - 1) / IB);
    const size_t sm = adj3_smem<TC, IB, AK>(op->n_angles);
    // opt in to more than 48 KB of shared memory when the buffers need it
    (void)smem_optin(op->ctx, (const void*)radon_adj3_kernel<TI, TO, TC, IB, AK>, sm);
    // a launch error is left for the caller's launch check (cudaGetLastError)
    (void)launch_pdl(radon_adj3_kernel<TI, TO, TC, IB, AK>, grid, 256, sm, op->ctx->stream, s, x, op->n1, op->n2,
                     op->n_angles, op->n_bins, nb, tables<TC>(op), (TC)((op->n1 - 1) / 2.0), (TC)((op->n2 - 1) / 2.0),
                     (TC)((op->n_bins - 1) / 2.0));
}

template <class TI, class TO, class TC>
int radon_adj(nys_op* op, const void* s, void* x, int batch) {
    // images per CTA: 4 for batches of 4 or more unless nys_op_autotune chose 1;
    // grid.z (images / ib) stays within 65535
    const int ib = (batch >= 4 && op->radon_adj_ib == 4) ? 4 : 1;
    for (int b0 = 0; b0 < batch; b0 += 65535 * ib) {
        const int nb = std::min(65535 * ib, batch - b0);
        const TI* sb = (const TI*)s + (size_t)b0 * op->M;
        TO* xb = (TO*)x + (size_t)b0 * op->N;
        // 4, 8 or 16 angles per round (nys_op_autotune)
        const int ak = op->radon_adj_ak;
        if (ib == 4 && nb >= 4) {
            if (ak == 4) radon_adj_launch<TI, TO, TC, 4, 4>(op, sb, xb, nb);
            else if (ak == 16) radon_adj_launch<TI, TO, TC, 4, 16>(op, sb, xb, nb);
            else radon_adj_launch<TI, TO, TC, 4, 8>(op, sb, xb, nb);
        } else {
            if (ak == 4) radon_adj_launch<TI, TO, TC, 1, 4>(op, sb, xb, nb);
            else if (ak == 16) radon_adj_launch<TI, TO, TC, 1, 16>(op, sb, xb, nb);
            else radon_adj_launch<TI, TO, TC, 1, 8>(op, sb, xb, nb);
        }
        NYS_LAUNCH_CK(op->ctx);
    }
    return NYS_OK;
}

template <class TI, class TO, class TC>
int radon_typed(nys_op* op, int which, const void* x, void* y, int batch) {
    if (which == 0) return radon_fwd<TI, TO, TC>(op, x, y, batch);
    if (which == 1) return radon_adj<TI, TO, TC>(op, x, y, batch);
    for (int b0 = 0; b0 < batch; b0 += op->chunk) {
        const int nb = std::min(op->chunk, batch - b0);
        if (int st = radon_fwd<TI, TC, TC>(op, (const TI*)x + (size_t)b0 * op->N, op->inter, nb)) return st;
        if (int st = radon_adj<TC, TO, TC>(op, op->inter, (TO*)y + (size_t)b0 * op->N, nb)) return st;
    }
    return NYS_OK;
}

}  // namespace

int radon_setup(nys_op* op) {
    const bool f64 = op->dtype == NYS_F64;
    int st = f64 ? build_tables<double>(op) : build_tables<float>(op);
    if (st) return st;
    op->chunk = 32;
    NYS_CK(op->ctx, cudaMalloc(&op->inter, (size_t)op->chunk * op->M * (f64 ? 8 : 4)));
    // line-major copies for the forward: transposed + row-major, `chunk` images
    NYS_CK(op->ctx, cudaMalloc(&op->lines, (size_t)2 * op->chunk * op->N * (f64 ? 8 : 4)));
    return NYS_OK;
}

int radon_run(nys_op* op, int which, const void* x, void* y, int batch, int in_dt, int out_dt) {
    if (op->dtype == NYS_F64) {
        if (in_dt != NYS_F64 || out_dt != NYS_F64) return fail(op->ctx, NYS_EINVAL, "f64 operator needs f64 data");
        return radon_typed<double, double, double>(op, which, x, y, batch);
    }
    const bool ib = in_dt == NYS_BF16, ob = out_dt == NYS_BF16;
    if (!ib && !ob) return radon_typed<float, float, float>(op, which, x, y, batch);
    if (ib && ob) return radon_typed<__nv_bfloat16, __nv_bfloat16, float>(op, which, x, y, batch);
    if (ib) return radon_typed<__nv_bfloat16, float, float>(op, which, x, y, batch);
    return radon_typed<float, __nv_bfloat16, float>(op, which, x, y, batch);
}

}  // namespace nys
