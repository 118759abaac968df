"""Matrix-free linear operators of the reconstruction problems (oracle side, float64).

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

Every function takes a batch of images with shape (..., n1, n2) -- pixel (i, j)
is row i, column j -- and is written as the plain definition, one term at a
time, so that it can be checked against the paper by eye.

  * blur (Sec. IV-A):  (Hx)[i,j] = sum_{a,b} h[a,b] x[(i+a-ch) mod n1, (j+b-cw) mod n2]
    with ch = (kh-1)/2, cw = (kw-1)/2 (correlation form, periodic boundary);
    H^T correlates with the flipped kernel.
  * blur + decimation (Sec. IV-A, super-resolution): A = D H with
    (Dz)[i,j] = z[d i, d j]; D^T zero-fills.
  * parallel-beam ray transform (Sec. IV-C, forward model of CT), discretised
    with Joseph's method (P. M. Joseph, IEEE TMI 1982): pixel (i, j) sits at
    x = j - (n2-1)/2, y = i - (n1-1)/2; ray (theta_k, t_m) is the line
    x cos(theta) + y sin(theta) = t with theta_k = k * span / n_angles and
    t_m = m - (n_bins-1)/2.  If |cos| + 1e-9 >= |sin| the ray is sampled once
    per row with linear interpolation between the two neighbouring columns and
    weight 1/|cos|; otherwise once per column with weight 1/|sin|.  Pixels
    outside the image are zero.  The adjoint is the exact transpose (same
    weights, scattered back).
  * orthonormal 2-D Haar transform W with the Mallat pyramid layout
    (the wavelet regulariser, Sec. III-B and IV-C).
  * first differences (Appendix A): v = (X[i,j]-X[i-1,j], X[i,j]-X[i,j-1]),
    periodic.
  * second differences (Appendix A): v11 = X[i-1,j]-2X[i,j]+X[i+1,j],
    v22 = X[i,j-1]-2X[i,j]+X[i,j+1],
    v12 = v21 = (X[i+1,j+1]-X[i+1,j-1]-X[i-1,j+1]+X[i-1,j-1])/4, periodic.
    Stored as (v11, v12, v22); the inner product on this space counts the
    off-diagonal entry twice (q11 v11 + 2 q12 v12 + q22 v22), so the adjoint
    carries a factor 2 on the cross term.
"""
from __future__ import annotations

import math

import numpy as np


# ----------------------------------------------------------------- blur ----

def blur_apply(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    kh, kw = h.shape
    ch, cw = (kh - 1) // 2, (kw - 1) // 2
    out = np.zeros_like(x)
    for a in range(kh):
        for b in range(kw):
            # x[(i + a - ch), (j + b - cw)] == roll by -(a-ch), -(b-cw)
            out += h[a, b] * np.roll(x, shift=(-(a - ch), -(b - cw)), axis=(-2, -1))
    return out


def blur_adjoint(y: np.ndarray, h: np.ndarray) -> np.ndarray:
    y = np.asarray(y, dtype=np.float64)
    kh, kw = h.shape
    ch, cw = (kh - 1) // 2, (kw - 1) // 2
    out = np.zeros_like(y)
    for a in range(kh):
        for b in range(kw):
            out += h[a, b] * np.roll(y, shift=(a - ch, b - cw), axis=(-2, -1))
    return out


# ------------------------------------------------------ blur + decimate ----

def decim_apply(x: np.ndarray, h: np.ndarray, d: int) -> np.ndarray:
    return blur_apply(x, h)[..., ::d, ::d]


def decim_adjoint(y: np.ndarray, h: np.ndarray, d: int) -> np.ndarray:
    y = np.asarray(y, dtype=np.float64)
    shape = y.shape[:-2] + (y.shape[-2] * d, y.shape[-1] * d)
    z = np.zeros(shape, dtype=np.float64)
    z[..., ::d, ::d] = y
    return blur_adjoint(z, h)


# ------------------------------------------------------------ ray transform

def radon_angles(n_angles: int, span: float = math.pi) -> np.ndarray:
    return np.arange(n_angles, dtype=np.float64) * (span / n_angles)


def _radon_rays(n1: int, n2: int, theta: float, n_bins: int):
    """Sample positions of all rays of one angle.

    Returns (rowstep, line_idx, lo_idx, w_lo, w_hi, weight) where for
    rowstep=True sample (r, m) interpolates X[r, lo] and X[r, lo+1]; for
    rowstep=False it interpolates X[lo, r] and X[lo+1, r].  Arrays are
    (n_lines, n_bins).
    """
    c1, c2 = (n1 - 1) / 2.0, (n2 - 1) / 2.0
    cb = (n_bins - 1) / 2.0
    t = np.arange(n_bins, dtype=np.float64) - cb
    cs, sn = math.cos(theta), math.sin(theta)
    if abs(cs) + 1e-9 >= abs(sn):
        y = np.arange(n1, dtype=np.float64) - c1
        u = (t[None, :] - y[:, None] * sn) / cs + c2
        lo = np.floor(u)
        w = u - lo
        return True, lo.astype(np.int64), 1.0 - w, w, 1.0 / abs(cs)
    x = np.arange(n2, dtype=np.float64) - c2
    v = (t[None, :] - x[:, None] * cs) / sn + c1
    lo = np.floor(v)
    w = v - lo
    return False, lo.astype(np.int64), 1.0 - w, w, 1.0 / abs(sn)


def radon_apply(x: np.ndarray, n_angles: int, n_bins: int, span: float = math.pi) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    n1, n2 = x.shape[-2:]
    lead = x.shape[:-2]
    out = np.zeros(lead + (n_angles, n_bins), dtype=np.float64)
    for k, th in enumerate(radon_angles(n_angles, span)):
        rowstep, lo, wlo, whi, wt = _radon_rays(n1, n2, th, n_bins)
        nl = lo.shape[0]
        line = np.broadcast_to(np.arange(nl)[:, None], lo.shape)
        lim = n2 if rowstep else n1
        acc = np.zeros(lead + (n_bins,), dtype=np.float64)
        for idx, wgt in ((lo, wlo), (lo + 1, whi)):
            ok = (idx >= 0) & (idx < lim)
            ii = np.where(ok, idx, 0)
            vals = x[..., line, ii] if rowstep else x[..., ii, line]
            acc += np.sum(np.where(ok, wgt, 0.0) * vals, axis=-2)
        out[..., k, :] = wt * acc
    return out


def radon_adjoint(s: np.ndarray, n1: int, n2: int, span: float = math.pi) -> np.ndarray:
    s = np.asarray(s, dtype=np.float64)
    n_angles, n_bins = s.shape[-2:]
    lead = s.shape[:-2]
    flat = s.reshape((-1, n_angles, n_bins))
    out = np.zeros((flat.shape[0], n1 * n2), dtype=np.float64)
    for k, th in enumerate(radon_angles(n_angles, span)):
        rowstep, lo, wlo, whi, wt = _radon_rays(n1, n2, th, n_bins)
        nl = lo.shape[0]
        line = np.broadcast_to(np.arange(nl)[:, None], lo.shape)
        lim = n2 if rowstep else n1
        for idx, wgt in ((lo, wlo), (lo + 1, whi)):
            ok = (idx >= 0) & (idx < lim)
            pix = (line * n2 + idx) if rowstep else (idx * n2 + line)
            pix = pix[ok]
            for b in range(flat.shape[0]):
                contrib = (wt * wgt * flat[b, k][None, :])[ok]
                out[b] += np.bincount(pix, weights=contrib, minlength=n1 * n2)
    return out.reshape(lead + (n1, n2))


# ---------------------------------------------------- fan-beam transform --
# A point source on a circle of radius R about the image centre and a flat
# detector at distance D from it (the fan-beam CT geometry): at angle theta,
# e_s = (cos, sin), e_d = (-sin, cos), source S = R e_s, detector centre
# S - D e_s, bin m at offset u_m = (m - (n_bins-1)/2) du along e_d; ray m runs
# from S to its bin.  Joseph's method per ray: a ray whose direction d has
# |d_y| >= |d_x| samples every row i at column position u = a + b i
# (b = d_x/d_y), weight |d|/|d_y|; otherwise every column j at row position
# u = a + b j (b = d_y/d_x), weight |d|/|d_x|; linear interpolation between
# floor(u) and floor(u) + 1, zero outside.  Pixel (i, j) sits at
# (j - c2, i - c1).

def fanbeam_tables(n1: int, n2: int, n_angles: int, n_bins: int, R: float, D: float, du: float,
                   span: float = 2.0 * math.pi):
    """Per ray (n_angles, n_bins): rowstep flag, a, b, weight."""
    c1, c2 = (n1 - 1) / 2.0, (n2 - 1) / 2.0
    th = np.arange(n_angles, dtype=np.float64)[:, None] * (span / n_angles)
    um = (np.arange(n_bins, dtype=np.float64)[None, :] - (n_bins - 1) / 2.0) * du
    cs, sn = np.cos(th), np.sin(th)
    Sx, Sy = R * cs, R * sn
    dx = -D * cs - um * sn
    dy = -D * sn + um * cs
    nd = np.sqrt(dx * dx + dy * dy)
    row = np.abs(dy) >= np.abs(dx)
    # the major component divides (never zero: |major| >= |d| / sqrt 2)
    major = np.where(row, dy, dx)
    minor = np.where(row, dx, dy)
    b = minor / major
    # row-step: u = Sx + (i - c1 - Sy) b + c2; column-step: u = Sy + (j - c2 - Sx) b + c1
    a = np.where(row, Sx - (c1 + Sy) * b + c2, Sy - (c2 + Sx) * b + c1)
    w = nd / np.abs(major)
    return row, a, b, w


def fanbeam_apply(x: np.ndarray, n_angles: int, n_bins: int, R: float, D: float, du: float,
                  span: float = 2.0 * math.pi) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    n1, n2 = x.shape[-2:]
    lead = x.shape[:-2]
    row, a, b, w = fanbeam_tables(n1, n2, n_angles, n_bins, R, D, du, span)
    out = np.zeros(lead + (n_angles, n_bins), dtype=np.float64)
    for k in range(n_angles):
        for rs, nl, lim in ((True, n1, n2), (False, n2, n1)):
            m = np.nonzero(row[k] == rs)[0]
            if m.size == 0:
                continue
            l = np.arange(nl, dtype=np.float64)
            u = a[k, m][:, None] + b[k, m][:, None] * l[None, :]        # (rays, lines)
            lo = np.floor(u)
            f = u - lo
            lo = lo.astype(np.int64)
            line = np.broadcast_to(np.arange(nl)[None, :], lo.shape)
            acc = np.zeros(lead + (m.size,), dtype=np.float64)
            for idx, wgt in ((lo, 1.0 - f), (lo + 1, f)):
                ok = (idx >= 0) & (idx < lim)
                ii = np.where(ok, idx, 0)
                vals = x[..., line, ii] if rs else x[..., ii, line]
                acc += np.sum(np.where(ok, wgt, 0.0) * vals, axis=-1)
            out[..., k, m] = w[k, m] * acc
    return out


def fanbeam_adjoint(s: np.ndarray, n1: int, n2: int, R: float, D: float, du: float,
                    span: float = 2.0 * math.pi) -> np.ndarray:
    s = np.asarray(s, dtype=np.float64)
    n_angles, n_bins = s.shape[-2:]
    lead = s.shape[:-2]
    flat = s.reshape((-1, n_angles, n_bins))
    row, a, b, w = fanbeam_tables(n1, n2, n_angles, n_bins, R, D, du, span)
    out = np.zeros((flat.shape[0], n1 * n2), dtype=np.float64)
    for k in range(n_angles):
        for rs, nl, lim in ((True, n1, n2), (False, n2, n1)):
            m = np.nonzero(row[k] == rs)[0]
            if m.size == 0:
                continue
            l = np.arange(nl, dtype=np.float64)
            u = a[k, m][:, None] + b[k, m][:, None] * l[None, :]
            lo = np.floor(u)
            f = u - lo
            lo = lo.astype(np.int64)
            line = np.broadcast_to(np.arange(nl)[None, :], lo.shape)
            for idx, wgt in ((lo, 1.0 - f), (lo + 1, f)):
                ok = (idx >= 0) & (idx < lim)
                pix = (line * n2 + idx) if rs else (idx * n2 + line)
                pix = pix[ok]
                for bb in range(flat.shape[0]):
                    contrib = (w[k, m][:, None] * wgt * flat[bb, k, m][:, None])[ok]
                    out[bb] += np.bincount(pix, weights=contrib, minlength=n1 * n2)
    return out.reshape(lead + (n1, n2))


# ------------------------------------------------------------------ Haar ---

_R2 = 1.0 / math.sqrt(2.0)


def haar_forward(x: np.ndarray, levels: int) -> np.ndarray:
    """Coefficients W x in the Mallat layout (low-low block top-left)."""
    c = np.array(x, dtype=np.float64, copy=True)
    h, w = c.shape[-2:]
    for _ in range(levels):
        blk = c[..., :h, :w]
        lo = (blk[..., :, 0::2] + blk[..., :, 1::2]) * _R2
        hi = (blk[..., :, 0::2] - blk[..., :, 1::2]) * _R2
        blk = np.concatenate([lo, hi], axis=-1)
        lo = (blk[..., 0::2, :] + blk[..., 1::2, :]) * _R2
        hi = (blk[..., 0::2, :] - blk[..., 1::2, :]) * _R2
        c[..., :h, :w] = np.concatenate([lo, hi], axis=-2)
        h, w = h // 2, w // 2
    return c


def haar_adjoint(c: np.ndarray, levels: int) -> np.ndarray:
    """W^T c, undoing the levels coarsest first (W is orthonormal)."""
    x = np.array(c, dtype=np.float64, copy=True)
    n1, n2 = x.shape[-2:]
    for lev in reversed(range(levels)):
        h, w = n1 >> lev, n2 >> lev
        blk = x[..., :h, :w]
        lo, hi = blk[..., : h // 2, :], blk[..., h // 2:, :]
        rows = np.empty_like(blk)
        rows[..., 0::2, :] = (lo + hi) * _R2
        rows[..., 1::2, :] = (lo - hi) * _R2
        lo, hi = rows[..., :, : w // 2], rows[..., :, w // 2:]
        cols = np.empty_like(blk)
        cols[..., :, 0::2] = (lo + hi) * _R2
        cols[..., :, 1::2] = (lo - hi) * _R2
        x[..., :h, :w] = cols
    return x


# ------------------------------------------- orthonormal filter banks ---
# A periodic two-channel orthonormal wavelet (Mallat's pyramid): one level
# along an axis of length n maps x to
#     lo[i] = sum_k h[k] x[(2 i + k) mod n],  hi[i] = sum_k g[k] x[(2 i + k) mod n],
# g[k] = (-1)^k h[L-1-k] (the quadrature-mirror high-pass), stored as [lo | hi];
# in 2-D the columns axis first, then the rows, and the next level works on
# the low-low block.  With h = (1, 1)/sqrt 2 this is the Haar transform above.
# Daubechies' four-tap filter (two vanishing moments, Daubechies 1988):
#     h = (1 + sqrt 3, 3 + sqrt 3, 3 - sqrt 3, 1 - sqrt 3) / (4 sqrt 2).

_S3 = math.sqrt(3.0)
WAVELET_TAPS = {
    "haar": np.array([1.0, 1.0]) / math.sqrt(2.0),
    "db4": np.array([1.0 + _S3, 3.0 + _S3, 3.0 - _S3, 1.0 - _S3]) / (4.0 * math.sqrt(2.0)),
}


def qmf_highpass(h: np.ndarray) -> np.ndarray:
    L = len(h)
    return np.array([(-1) ** k * h[L - 1 - k] for k in range(L)])


def _analysis(x, h, axis):
    g = qmf_highpass(h)
    n = x.shape[axis]
    i2 = 2 * np.arange(n // 2)
    lo = sum(h[k] * np.take(x, (i2 + k) % n, axis=axis) for k in range(len(h)))
    hi = sum(g[k] * np.take(x, (i2 + k) % n, axis=axis) for k in range(len(h)))
    return np.concatenate([lo, hi], axis=axis)


def _synthesis(c, h, axis):
    # the transpose of _analysis: x[(2 i + k) mod n] += h[k] lo[i] + g[k] hi[i]
    g = qmf_highpass(h)
    n = c.shape[axis]
    lo, hi = np.split(c, 2, axis=axis)
    x = np.zeros_like(c)
    i2 = 2 * np.arange(n // 2)
    for k in range(len(h)):
        idx = (i2 + k) % n
        contrib = h[k] * lo + g[k] * hi
        xm = np.moveaxis(x, axis, 0)
        np.add.at(xm, idx, np.moveaxis(contrib, axis, 0))
    return x


def wavelet_forward(x: np.ndarray, levels: int, kind: str = "haar") -> np.ndarray:
    """Coefficients W x in the Mallat layout for the filter bank `kind`."""
    h = WAVELET_TAPS[kind]
    c = np.array(x, dtype=np.float64, copy=True)
    hh, ww = c.shape[-2:]
    for _ in range(levels):
        blk = _analysis(c[..., :hh, :ww], h, axis=-1)
        c[..., :hh, :ww] = _analysis(blk, h, axis=-2)
        hh, ww = hh // 2, ww // 2
    return c


def wavelet_adjoint(c: np.ndarray, levels: int, kind: str = "haar") -> np.ndarray:
    """W^T c (= W^{-1} c, W orthonormal), coarsest level first."""
    h = WAVELET_TAPS[kind]
    x = np.array(c, dtype=np.float64, copy=True)
    n1, n2 = x.shape[-2:]
    for lev in reversed(range(levels)):
        hh, ww = n1 >> lev, n2 >> lev
        blk = _synthesis(x[..., :hh, :ww], h, axis=-2)
        x[..., :hh, :ww] = _synthesis(blk, h, axis=-1)
    return x


# ----------------------------------------------- finite differences --------

def grad(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    v1 = x - np.roll(x, 1, axis=-2)          # X[i,j] - X[i-1,j]
    v2 = x - np.roll(x, 1, axis=-1)          # X[i,j] - X[i,j-1]
    return np.stack([v1, v2], axis=-3)


def grad_adjoint(q: np.ndarray) -> np.ndarray:
    q1, q2 = q[..., 0, :, :], q[..., 1, :, :]
    return (q1 - np.roll(q1, -1, axis=-2)) + (q2 - np.roll(q2, -1, axis=-1))


def _sh(x, di, dj):
    """X[i+di, j+dj] (periodic)."""
    return np.roll(x, shift=(-di, -dj), axis=(-2, -1))


def hess(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    v11 = _sh(x, -1, 0) - 2.0 * x + _sh(x, 1, 0)
    v22 = _sh(x, 0, -1) - 2.0 * x + _sh(x, 0, 1)
    v12 = 0.25 * (_sh(x, 1, 1) - _sh(x, 1, -1) - _sh(x, -1, 1) + _sh(x, -1, -1))
    return np.stack([v11, v12, v22], axis=-3)


def hess_adjoint(q: np.ndarray) -> np.ndarray:
    """Adjoint for the inner product q11 v11 + 2 q12 v12 + q22 v22."""
    q11, q12, q22 = q[..., 0, :, :], q[..., 1, :, :], q[..., 2, :, :]
    # each stencil is symmetric under (di, dj) -> (-di, -dj)
    a11 = _sh(q11, -1, 0) - 2.0 * q11 + _sh(q11, 1, 0)
    a22 = _sh(q22, 0, -1) - 2.0 * q22 + _sh(q22, 0, 1)
    a12 = 0.25 * (_sh(q12, 1, 1) - _sh(q12, 1, -1) - _sh(q12, -1, 1) + _sh(q12, -1, -1))
    return a11 + 2.0 * a12 + a22


HESS_WEIGHTS = np.array([1.0, 2.0, 1.0])


# ----------------------------------------------------- operator wrapper ----

class Operator:
    """A forward model A with its exact adjoint, on (..., n1, n2) images."""

    def __init__(self, kind: str, n1: int, n2: int, kernel=None, decim: int = 1,
                 n_angles: int = 0, n_bins: int = 0, span: float | None = None,
                 src_dist: float = 0.0, det_dist: float = 0.0, det_spacing: float = 1.0):
        self.kind, self.n1, self.n2 = kind, n1, n2
        self.kernel = None if kernel is None else np.asarray(kernel, dtype=np.float64)
        if span is None:
            span = 2.0 * math.pi if kind == "fanbeam" else math.pi
        self.decim, self.n_angles, self.n_bins, self.span = decim, n_angles, n_bins, span
        self.R, self.D, self.du = src_dist, det_dist, det_spacing
        if kind == "blur":
            self.meas_shape = (n1, n2)
        elif kind == "blur_decim":
            self.meas_shape = (n1 // decim, n2 // decim)
        elif kind in ("radon", "fanbeam"):
            self.meas_shape = (n_angles, n_bins)
        else:
            raise ValueError(kind)

    def apply(self, x):
        if self.kind == "blur":
            return blur_apply(x, self.kernel)
        if self.kind == "blur_decim":
            return decim_apply(x, self.kernel, self.decim)
        if self.kind == "fanbeam":
            return fanbeam_apply(x, self.n_angles, self.n_bins, self.R, self.D, self.du, self.span)
        return radon_apply(x, self.n_angles, self.n_bins, self.span)

    def adjoint(self, y):
        if self.kind == "blur":
            return blur_adjoint(y, self.kernel)
        if self.kind == "blur_decim":
            return decim_adjoint(y, self.kernel, self.decim)
        if self.kind == "fanbeam":
            return fanbeam_adjoint(y, self.n1, self.n2, self.R, self.D, self.du, self.span)
        return radon_adjoint(y, self.n1, self.n2, self.span)

    def normal(self, x):
        """A^T A x."""
        return self.adjoint(self.apply(x))
