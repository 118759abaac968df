"""Host-side checks of the index logic the fan-beam adjoint relies on,
restated in numpy from the flat-detector Joseph geometry (float64 ray tables
as the host builds them, the float32-rounded angle table the kernel reads):

* a pixel gathers, per angle, only the bins between the detector
  coordinates of its two neighbours along the ray's stepping axis, widened by
  one bin; every ray whose interpolation touches the pixel with a nonzero
  weight must lie in that range (it crosses the pixel's row or column within
  one pixel of it, and the detector coordinate is monotone along that
  segment) -- a ray outside it would be dropped silently;
* a pixel tries row-step rays only when |v_y| >= |v_x| (1 - 8/depth) and
  column-step rays only when |v_x| >= |v_y| (1 - 8/depth), v the vector from
  the source to the pixel: every touching ray must pass the test of its kind;
* the source is validated to lie more than two pixels beyond the image's
  half-diagonal, so every point the kernel projects (pixel centres and their
  neighbours) has depth above one pixel and the divisions are safe.
"""
import math

import numpy as np
import pytest

MARGIN_BINS = 1.0       # the kernel's widening of the candidate range
KIND_TOL = 8.0          # the kernel's ray-kind tolerance, divided by the depth


def tables(n1, n2, A, B, R, D, du, span=2 * math.pi):
    c1, c2, cb = (n1 - 1) / 2, (n2 - 1) / 2, (B - 1) / 2
    th = np.arange(A) * (span / A)
    cs, sn = np.cos(th)[:, None], np.sin(th)[:, None]
    Sx, Sy = R * cs, R * sn
    um = ((np.arange(B) - cb) * du)[None, :]
    dx, dy = -D * cs - um * sn, -D * sn + um * cs
    row = np.abs(dy) >= np.abs(dx)
    major, minor = np.where(row, dy, dx), np.where(row, dx, dy)
    b = minor / major
    a = np.where(row, Sx - (c1 + Sy) * b + c2, Sy - (c2 + Sx) * b + c1)
    ang = np.stack([R * np.cos(th), R * np.sin(th), np.cos(th), np.sin(th)], 1).astype(np.float32)
    return a, b, row, ang.astype(np.float64)


def touching(a, b, row, k, kind, n1, n2):
    """(bin, pixel row, pixel column) of every nonzero interpolation weight of
    angle k's rays of one kind (0: row-step, 1: column-step)."""
    sel = np.nonzero(row[k] == (kind == 0))[0]
    nl, na = (n1, n2) if kind == 0 else (n2, n1)
    l = np.arange(nl)[None, :]
    u = b[k, sel][:, None] * l + a[k, sel][:, None]
    lo = np.floor(u)
    f = u - lo
    out = []
    for p, w in ((lo, 1 - f), (lo + 1, f)):
        mi, li = np.nonzero((p >= 0) & (p < na) & (w > 1e-9))
        pp = p[mi, li].astype(np.int64)
        out.append((sel[mi], li, pp) if kind == 0 else (sel[mi], pp, li))
    return [np.concatenate(c) for c in zip(*out)]


def margins(n1, n2, A, B, R, D, du, angles):
    """Largest excess of a touching bin beyond the neighbours' detector range
    (bins), largest share of the kind tolerance a touching ray needs, smallest
    depth of a projected point, number of touching (ray, pixel) pairs."""
    a, b, row, ang = tables(n1, n2, A, B, R, D, du)
    c1, c2, cb = (n1 - 1) / 2, (n2 - 1) / 2, (B - 1) / 2
    worst_bin, worst_kind, min_depth, hits = -np.inf, 0.0, np.inf, 0
    for k in angles:
        Sx, Sy, cs, sn = ang[k]

        def depth_bin(qx, qy):
            vx, vy = qx - Sx, qy - Sy
            depth = -(vx * cs + vy * sn)
            return depth, D * (-vx * sn + vy * cs) / depth / du + cb

        for kind in (0, 1):
            m, i, j = touching(a, b, row, k, kind, n1, n2)
            if m.size == 0:
                continue
            px, py = j - c2, i - c1
            e1, e2 = ((-1, 0), (1, 0)) if kind == 0 else ((0, -1), (0, 1))
            d1, m1 = depth_bin(px + e1[0], py + e1[1])
            d2, m2 = depth_bin(px + e2[0], py + e2[1])
            d0, _ = depth_bin(px, py)
            min_depth = min(min_depth, d0.min(), d1.min(), d2.min())
            worst_bin = max(worst_bin, np.maximum(np.minimum(m1, m2) - m, m - np.maximum(m1, m2)).max())
            vx, vy = np.abs(px - Sx), np.abs(py - Sy)
            major, minor = (vy, vx) if kind == 0 else (vx, vy)
            # the test passes iff minor - major <= minor * tol
            need = np.where(minor > 0, (minor - major) / np.where(minor > 0, minor, 1.0), 0.0) / (KIND_TOL / d0)
            worst_kind = max(worst_kind, need.max())
            hits += m.size
    return worst_bin, worst_kind, min_depth, hits


def _limit_R(n1, n2):
    return 0.5 * math.hypot(n1, n2) + 2.0 + 1e-6      # just inside the validated geometry


@pytest.mark.parametrize("n1,n2,A,B,R,D,du", [
    (16, 16, 12, 40, 30.0, 60.0, 1.0),
    (20, 28, 17, 61, 25.0, 55.0, 0.75),
    (24, 24, 9, 30, None, 40.0, 1.0),
    (64, 64, 90, 160, 50.0, 100.0, 1.0),
    (128, 96, 180, 256, 83.0, 160.0, 1.3),
])
def test_fanbeam_adjoint_candidates_cover_every_touching_ray(n1, n2, A, B, R, D, du):
    R = _limit_R(n1, n2) if R is None else R
    worst_bin, worst_kind, min_depth, hits = margins(n1, n2, A, B, R, D, du, range(A))
    assert hits > 1000
    # geometrically every touching bin lies in the neighbours' range; float32
    # angles move it by far less than the kernel's margin
    assert worst_bin <= 0.25 * MARGIN_BINS, worst_bin
    assert worst_kind <= 0.5, worst_kind
    assert min_depth > 1.0, min_depth


def test_fanbeam_adjoint_candidates_at_the_measured_size():
    # 512^2, 720 angles over the full circle, 1024 bins, R = 1000, D = 2000:
    # every 30th angle and the angles around the axis-aligned views
    A = 720
    angles = sorted(set(range(0, A, 30)) | {89, 90, 91, 179, 180, 181, 269, 270, 271, 359, 360, 361})
    worst_bin, worst_kind, min_depth, hits = margins(512, 512, A, 1024, 1000.0, 2000.0, 1.0, angles)
    assert hits > 10 ** 7
    assert worst_bin <= 0.25 * MARGIN_BINS, worst_bin
    assert worst_kind <= 0.5, worst_kind
    assert min_depth > 1.0, min_depth


def split_positions(a, b, row, n1, n2):
    """The float32 operators' positions, restated in numpy float32 from the
    host's split (integer + fraction about the middle line l0, b = bhi + blo
    with bhi on a 2^-12 grid): returns (integer part, fraction) of every ray on
    every line l < max(n1, n2) (lines past a ray's own count are ignored)."""
    L = max(n1, n2)
    l0 = np.where(row, n1 // 2, n2 // 2)
    bhi = np.round(b * 4096.0) / 4096.0
    am = a + b * l0
    ai = np.floor(am)
    sp_x, sp_y = ai.astype(np.float32), (am - ai).astype(np.float32)
    sp_z, sp_w = bhi.astype(np.float32), (b - bhi).astype(np.float32)
    k = (np.arange(L)[None, None, :] - l0[..., None]).astype(np.float32)
    t = sp_z[..., None] * k
    ft = np.floor(t)
    fr = (sp_w[..., None] * k).astype(np.float64) + (sp_y[..., None] + (t - ft)).astype(np.float64)
    fr = fr.astype(np.float32)   # a fused multiply-add rounds once: emulate it in float64, round at the end
    ff = np.floor(fr)
    return (sp_x[..., None] + ft + ff).astype(np.float64), (fr - ff).astype(np.float64)


@pytest.mark.parametrize("geom", [(24, 24, 9, 40, 30.0, 60.0, 1.0), (20, 28, 7, 47, 30.0, 60.0, 1.0),
                                  (512, 512, 24, 1024, 1000.0, 2000.0, 1.0)])
def test_float32_split_positions_match_float64(geom):
    # the float32 evaluation agrees with u = a + b l to 1e-6 of a pixel, so
    # its interpolation weights agree with the float64 (oracle) ones to 1e-6
    n1, n2, A, B, R, D, du = geom
    a, b, row, _ = tables(n1, n2, A, B, R, D, du)
    ip, fr = split_positions(a, b, row, n1, n2)
    L = max(n1, n2)
    u = a[..., None] + b[..., None] * np.arange(L)[None, None, :]
    err = np.abs((ip + fr) - u)
    assert err.max() < 1e-6, err.max()
    assert np.all((fr >= 0.0) & (fr < 1.0))
