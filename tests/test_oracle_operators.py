"""Pins for the oracle's operators against closed forms and invariants."""
import math

import numpy as np
import pytest

from oracle import operators as ops
from workloads import gaussian_kernel, random_kernel


def dense(fn, shape_in):
    """Matrix of a linear map given on arrays of shape shape_in."""
    n = int(np.prod(shape_in))
    eye = np.eye(n).reshape((n,) + tuple(shape_in))
    return fn(eye).reshape(n, -1).T


def dot_test(A, At, xshape, yshape, seed=0, w=None):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(xshape)
    y = rng.standard_normal(yshape)
    Ax = A(x)
    lhs = np.sum((Ax * (w if w is not None else 1.0)) * y)
    rhs = np.sum(x * At(y))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, np.linalg.norm(Ax) * np.linalg.norm(y))


# ----------------------------------------------------------------- blur ----

def test_blur_delta_gives_flipped_kernel_centred():
    n = 16
    h = random_kernel(5, seed=1)
    x = np.zeros((n, n))
    x[8, 8] = 1.0
    y = ops.blur_apply(x, h)
    # (Hx)[i,j] = h[a,b] where 8 = i + a - 2, 8 = j + b - 2 -> a = 10 - i
    expect = np.zeros((n, n))
    for a in range(5):
        for b in range(5):
            expect[10 - a, 10 - b] = h[a, b]
    assert np.allclose(y, expect, atol=1e-15)


def test_blur_constant_and_wraparound():
    h = gaussian_kernel(9, 1.5)
    x = np.full((12, 12), 3.25)
    assert np.allclose(ops.blur_apply(x, h), 3.25, atol=1e-13)
    # periodic: a delta at the corner spreads to all four corners
    x = np.zeros((12, 12))
    x[0, 0] = 1.0
    y = ops.blur_apply(x, h)
    assert y[11, 11] > 0 and y[1, 1] > 0 and abs(y.sum() - 1.0) < 1e-13


def test_blur_normal_spectrum_is_dft_closed_form():
    # H^T H is block-circulant: its eigenvalues are |DFT2(h placed on the grid)|^2
    n = 8
    h = random_kernel(3, seed=4)
    M = dense(lambda x: ops.blur_adjoint(ops.blur_apply(x, h), h), (n, n))
    ev = np.sort(np.linalg.eigvalsh(0.5 * (M + M.T)))
    pad = np.zeros((n, n))
    for a in range(3):
        for b in range(3):
            pad[(a - 1) % n, (b - 1) % n] = h[a, b]
    sym = np.sort(np.abs(np.fft.fft2(pad)).ravel() ** 2)
    assert np.allclose(ev, sym, atol=1e-12)


@pytest.mark.parametrize("k", [3, 5, 9])
def test_blur_adjoint_dot(k):
    h = random_kernel(k, seed=k)
    dot_test(lambda x: ops.blur_apply(x, h), lambda y: ops.blur_adjoint(y, h), (2, 20, 18), (2, 20, 18))


def test_decim_adjoint_and_selection():
    h = gaussian_kernel(7, 2.0)
    dot_test(lambda x: ops.decim_apply(x, h, 4), lambda y: ops.decim_adjoint(y, h, 4), (3, 16, 16), (3, 4, 4))
    x = np.random.default_rng(0).standard_normal((16, 16))
    assert np.allclose(ops.decim_apply(x, h, 4), ops.blur_apply(x, h)[::4, ::4])
    # D D^T = I
    y = np.random.default_rng(1).standard_normal((4, 4))
    d = np.eye(1)[0, 0]
    assert np.allclose(ops.decim_apply(ops.decim_adjoint(y, np.array([[d]]), 4), np.array([[d]]), 4), y)


# ------------------------------------------------------------------ Haar ---

def test_haar_orthonormal_dense():
    W = dense(lambda x: ops.haar_forward(x, 3), (8, 8))
    assert np.allclose(W.T @ W, np.eye(64), atol=1e-13)
    Wt = dense(lambda c: ops.haar_adjoint(c, 3), (8, 8))
    assert np.allclose(Wt, W.T, atol=1e-13)


def test_haar_one_level_2x2_closed_form():
    a, b, c, d = 1.0, 2.0, 5.0, 11.0
    x = np.array([[a, b], [c, d]])
    w = ops.haar_forward(x, 1)
    # averages/differences of the four values, orthonormal scaling 1/2
    assert np.allclose(w, 0.5 * np.array([[a + b + c + d, a - b + c - d],
                                          [a + b - c - d, a - b - c + d]]))


def test_haar_constant_image_only_coarse_coefficients():
    x = np.full((16, 16), 2.0)
    w = ops.haar_forward(x, 3)
    assert np.allclose(w[:2, :2], 2.0 * 8)           # 2 * (2*2*2) per coarse coeff
    w[:2, :2] = 0.0
    assert np.allclose(w, 0.0)
    assert np.isclose(np.linalg.norm(ops.haar_forward(np.arange(256.0).reshape(16, 16), 3)),
                      np.linalg.norm(np.arange(256.0)))


# --------------------------------------------------- finite differences ---

def test_grad_ramp_values():
    n = 6
    X = np.tile(np.arange(n, dtype=float)[:, None], (1, n))   # X[i,j] = i
    v = ops.grad(X)
    expect1 = np.ones((n, n))
    expect1[0, :] = -(n - 1)                                   # periodic wrap
    assert np.allclose(v[0], expect1) and np.allclose(v[1], 0.0)


def test_hessian_polynomial_values():
    n = 10
    i = np.arange(n, dtype=float)[:, None]
    j = np.arange(n, dtype=float)[None, :]
    v = ops.hess(i * j + 0.0 * j)
    inner = (slice(1, n - 1), slice(1, n - 1))
    assert np.allclose(v[1][inner], 1.0)                       # d2/dxdy (ij) = 1
    assert np.allclose(v[0][inner], 0.0) and np.allclose(v[2][inner], 0.0)
    v = ops.hess(i * i + 0.0 * j)
    assert np.allclose(v[0][inner], 2.0) and np.allclose(v[2][inner], 0.0)


def test_difference_adjoints():
    dot_test(ops.grad, ops.grad_adjoint, (2, 7, 9), (2, 2, 7, 9))
    w = ops.HESS_WEIGHTS[:, None, None]
    dot_test(ops.hess, ops.hess_adjoint, (7, 9), (3, 7, 9), w=w)


def test_difference_norms():
    n = 8
    G = dense(ops.grad, (n, n))
    assert np.isclose(np.linalg.norm(G, 2) ** 2, 8.0)
    Hm = dense(ops.hess, (n, n))
    wts = np.repeat(ops.HESS_WEIGHTS, n * n)
    HtWH = Hm.T @ (wts[:, None] * Hm)
    assert np.isclose(np.linalg.eigvalsh(HtWH).max(), 32.0)
    # symbol of the first differences: (2-2cos w1) + (2-2cos w2)
    ev = np.sort(np.linalg.eigvalsh(G.T @ G))
    w = 2 * np.pi * np.arange(n) / n
    sym = np.sort(((2 - 2 * np.cos(w))[:, None] + (2 - 2 * np.cos(w))[None, :]).ravel())
    assert np.allclose(ev, sym, atol=1e-12)


# -------------------------------------------------------- ray transform ---

def test_radon_zero_angle_is_column_sums():
    n, nb = 16, 24
    x = np.random.default_rng(0).uniform(size=(n, n))
    s = ops.radon_apply(x, 4, nb)          # angles 0, 45, 90, 135 degrees
    cb = (nb - 1) / 2.0
    c = (n - 1) / 2.0
    col = {int(round(m - cb + c)): m for m in range(nb)}
    for j in range(n):
        assert np.isclose(s[0, col[j]], x[:, j].sum(), atol=1e-12)
    # 90 degrees: ray x*0 + y*1 = t -> row sums
    for i in range(n):
        assert np.isclose(s[2, col[i]], x[i, :].sum(), atol=1e-12)


def test_radon_disk_chords():
    n, nb, r = 96, 140, 30.0
    c = (n - 1) / 2.0
    ii, jj = np.meshgrid(np.arange(n) - c, np.arange(n) - c, indexing="ij")
    # supersampled area fraction of a disk
    sub = np.zeros((n, n))
    for dy in np.linspace(-0.375, 0.375, 4):
        for dx in np.linspace(-0.375, 0.375, 4):
            sub += ((ii + dy) ** 2 + (jj + dx) ** 2 <= r * r)
    x = sub / 16.0
    s = ops.radon_apply(x, 7, nb)
    t = np.arange(nb) - (nb - 1) / 2.0
    chord = 2.0 * np.sqrt(np.maximum(r * r - t * t, 0.0))
    for k in range(7):
        err = np.abs(s[k] - chord).sum() / chord.sum()
        assert err < 0.02, (k, err)
        assert abs(s[k].sum() - x.sum()) / x.sum() < 0.01


def test_radon_adjoint_dot():
    dot_test(lambda x: ops.radon_apply(x, 9, 17), lambda y: ops.radon_adjoint(y, 12, 10, math.pi),
             (2, 12, 10), (2, 9, 17))
