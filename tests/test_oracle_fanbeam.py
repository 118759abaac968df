"""Pins for the oracle's fan-beam Joseph projector (flat detector, point
source on a circle):

* the adjoint, written as a separate scatter, is the transpose of the
  forward (dot-product test);
* a constant image projects to the chord length of each ray through the
  pixel-edge square, up to the one-pixel interpolation ramps at the edges
  the ray steps across;
* a single bright pixel lights exactly the bins whose rays pass within one
  pixel of it, around the detector coordinate of its centre seen from the
  source;
* with the source far away the fan becomes parallel: the projection agrees
  with the parallel-beam transform of the quarter-turned image, to first
  order in image size / source distance.
"""
import math

import numpy as np
import pytest

from oracle import operators as ops


def _chord(S, d, half1, half2):
    """Length of the segment of the line S + t d inside |x| <= half2, |y| <= half1 (slab method)."""
    t0, t1 = -np.inf, np.inf
    for s0, dd, h in ((S[0], d[0], half2), (S[1], d[1], half1)):
        if abs(dd) < 1e-15:
            if abs(s0) > h:
                return 0.0
            continue
        a, b = (-h - s0) / dd, (h - s0) / dd
        t0, t1 = max(t0, min(a, b)), min(t1, max(a, b))
    return max(0.0, t1 - t0) * math.hypot(d[0], d[1])


@pytest.mark.parametrize("n1,n2,A,B", [(16, 16, 9, 40), (12, 20, 7, 33)])
def test_fanbeam_adjoint_dot(n1, n2, A, B):
    rng = np.random.default_rng(0)
    x = rng.standard_normal((n1, n2))
    y = rng.standard_normal((A, B))
    R, D, du = 30.0, 60.0, 1.0
    lhs = np.sum(ops.fanbeam_apply(x, A, B, R, D, du) * y)
    rhs = np.sum(x * ops.fanbeam_adjoint(y, n1, n2, R, D, du))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_fanbeam_constant_image_gives_chord_lengths():
    # Joseph's interpolation along a line turns the pixel edges the line
    # steps across into ramps one pixel wide: a ray crossing such an edge at
    # slope t (pixels across per line) spends about 1/t lines in the ramp, so
    # the projection matches the chord through the pixel-edge square to
    # within (2 + 1/t) line steps of the ray (vacuous only for rays running
    # along an edge)
    n, A, B, R, D, du = 24, 11, 61, 40.0, 80.0, 1.0
    p = ops.fanbeam_apply(np.ones((n, n)), A, B, R, D, du)
    half = n / 2.0
    checked = 0
    for k in range(A):
        th = k * 2 * math.pi / A
        S = (R * math.cos(th), R * math.sin(th))
        for m in range(B):
            um = (m - (B - 1) / 2.0) * du
            d = (-D * math.cos(th) - um * math.sin(th), -D * math.sin(th) + um * math.cos(th))
            major, minor = max(abs(d[0]), abs(d[1])), min(abs(d[0]), abs(d[1]))
            step = math.hypot(d[0], d[1]) / major        # path length per line
            slope = minor / major
            c = _chord(S, d, half, half)
            tol = step * (2.0 + min(n, 1.0 / max(slope, 1e-12)))
            assert abs(p[k, m] - c) <= tol + 1e-9, (k, m, p[k, m], c)
            checked += slope > 0.2 and c > 0
    assert checked > 100


def test_fanbeam_single_pixel_lights_the_expected_bins():
    n, A, B, R, D, du = 20, 6, 81, 35.0, 70.0, 0.5
    i0, j0 = 6, 13
    x = np.zeros((n, n))
    x[i0, j0] = 1.0
    p = ops.fanbeam_apply(x, A, B, R, D, du)
    c = (n - 1) / 2.0
    P = np.array([j0 - c, i0 - c])
    for k in range(A):
        th = k * 2 * math.pi / A
        es, ed = np.array([math.cos(th), math.sin(th)]), np.array([-math.sin(th), math.cos(th)])
        S = R * es
        v = P - S
        u_star = D * np.dot(v, ed) / np.dot(v, -es)      # detector coordinate of the pixel centre
        m_star = u_star / du + (B - 1) / 2.0
        lit = np.nonzero(p[k] > 0)[0]
        assert lit.size > 0
        # a ray samples the pixel only if it passes within one pixel of its
        # centre; at the pixel's depth one pixel spans (D / depth) / du bins
        depth = np.dot(v, -es)
        reach = math.sqrt(2.0) * (D / depth) / du + 1.0
        assert np.all(np.abs(lit - m_star) <= reach), (k, lit, m_star)
        assert int(round(m_star)) in lit


def test_fanbeam_far_source_tends_to_parallel_beam():
    n, A, B = 16, 5, 41
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (n, n))
    R = 1e7
    fan = ops.fanbeam_apply(x, A, B, R, 2 * R, 2.0, span=math.pi)    # magnification 2, unit bins at the centre
    # fan angle theta has rays along e_s, a quarter turn from the parallel
    # rays of angle theta (direction (-sin, cos)): the parallel transform of
    # the image turned by a quarter (np.rot90), same bin order
    par = ops.radon_apply(np.rot90(x, k=1), A, B, span=math.pi)
    assert np.abs(fan - par).max() <= 1e-4 * np.abs(par).max()
