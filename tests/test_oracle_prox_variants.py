"""Pins for the oracle's other mixed-norm regularisers of Eq. lpl1qMixedNorm:
isotropic TV (phi = 2 on each pixel's gradient pair) and the Hessian
Schatten-2 and Schatten-inf norms, alongside the anisotropic TV and HS_1 the
hot path uses.

* each dual-ball projection returns the nearest point of its ball (checked
  against dense random sampling of the ball in the same metric);
* on an image that varies along one axis only, every first-order variant
  gives the same prox, and so does every Hessian variant (the second
  component of the gradient, and the cross and second diagonal Hessian terms,
  vanish, and all balls then reduce to the interval [-1, 1]);
* the dual APG closes the duality gap of the prox problem, which ties each
  projection to the primal norm that reg_value evaluates (a ball of the wrong
  norm would leave a gap).
"""
import numpy as np
import pytest

from oracle import nystrom as ny
from oracle import operators as ops
from oracle import prox as px


def _weighted_dist2(p, q, w):
    return np.sum(w * (p - q) ** 2, axis=-1)


@pytest.mark.parametrize("name", ["isotv", "hs2", "hsinf", "hs"])
def test_projection_is_nearest_point_of_the_ball(name):
    rng = np.random.default_rng(1)
    G = px.DUAL_COMPONENTS[name]
    w = np.ones(G) if G == 2 else np.array([1.0, 2.0, 1.0])   # metric of the dual space

    def norm(v):      # the dual-ball norm of vectors v (..., G)
        if name == "isotv":
            return np.sqrt(v[..., 0] ** 2 + v[..., 1] ** 2)
        a, b, c = v[..., 0], v[..., 1], v[..., 2]
        m, r = 0.5 * (a + c), np.sqrt((0.5 * (a - c)) ** 2 + b * b)
        if name == "hs2":
            return np.sqrt(a * a + 2 * b * b + c * c)
        if name == "hsinf":
            return np.abs(m + r) + np.abs(m - r)           # Schatten-1
        return np.maximum(np.abs(m + r), np.abs(m - r))   # spectral (HS_1's dual ball)

    proj = px.REGULARISERS[name][3]
    q = rng.normal(0.0, 1.2, (40, G))
    p = proj(q.T.reshape(G, 40, 1)).reshape(G, 40).T
    assert np.all(norm(p) <= 1.0 + 1e-12)
    pp = proj(p.T.reshape(G, 40, 1)).reshape(G, 40).T
    assert np.allclose(pp, p, atol=1e-14)                 # idempotent
    inside = norm(q) <= 1.0
    assert np.allclose(p[inside], q[inside], atol=1e-15)
    # dense sample of the ball: nothing is closer to q than p
    cand = rng.uniform(-1.0, 1.0, (400000, G))
    if G == 3:
        cand[:, 1] *= 0.75
    cand = cand[norm(cand) <= 1.0]
    for i in range(q.shape[0]):
        d_best = _weighted_dist2(cand, q[i], w).min()
        assert _weighted_dist2(p[i], q[i], w) <= d_best + 1e-12, (name, i)


@pytest.mark.parametrize("group", [("tv", "isotv"), ("hs", "hs2", "hsinf")])
def test_variants_agree_on_a_one_axis_image(group):
    rng = np.random.default_rng(2)
    n1, n2 = 12, 9
    s = np.repeat(rng.uniform(0, 1, (n1, 1)), n2, axis=1)   # varies along rows only
    P = ny.Identity()
    xs = [px.prox_dual(s, reg, 0.05, P, 40)[0] for reg in group]
    for x in xs[1:]:
        assert np.abs(x - xs[0]).max() <= 1e-13
    vals = [px.reg_value(xs[0], reg) for reg in group]
    assert np.allclose(vals, vals[0], rtol=1e-12)


@pytest.mark.parametrize("reg", ["tv", "isotv", "hs", "hs2", "hsinf"])
def test_dual_apg_closes_the_duality_gap(reg):
    rng = np.random.default_rng(3)
    s = rng.uniform(0, 1, (10, 12))
    lb = 0.05
    L, Lt, _, proj = px.REGULARISERS[reg]
    x, Q = px.prox_dual(s, reg, lb, ny.Identity(), 4000)
    assert np.abs(proj(Q) - Q).max() <= 1e-12              # Q in the dual ball
    primal = 0.5 * np.sum((x - s) ** 2) + lb * px.reg_value(x, reg)
    dual = 0.5 * np.sum(s ** 2) - 0.5 * np.sum((s - lb * Lt(Q)) ** 2)
    assert -1e-12 <= primal - dual <= 1e-7 * primal, (reg, primal, dual)


def test_isotropic_value_is_euclidean_gradient_norm():
    # a linear ramp x = i + 2 j has gradient (1, 2) away from the wrap-around
    n = 8
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = (i + 2.0 * j).astype(float)
    g = ops.grad(x)
    interior = (i > 0) & (j > 0)
    assert np.allclose(g[0][interior], 1.0) and np.allclose(g[1][interior], 2.0)
    iso = np.sqrt(g[0] ** 2 + g[1] ** 2)
    assert px.reg_value(x, "isotv") == pytest.approx(iso.sum())
    assert np.allclose(iso[interior], np.sqrt(5.0))
