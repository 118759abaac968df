"""Pins for the oracle's unrolled-solve gradient (d MSE / d lambda, d MSE / d h).

The hand-derived reverse pass is checked against central finite differences of
the forward map in float64, and against PyTorch autograd (float64, CPU) run on
an independent re-statement of the same forward iteration.  The forward itself
is checked against Algorithm 3 as the oracle's WAPG computes it.
"""
import math

import numpy as np
import pytest

from oracle import nystrom as ny
from oracle import operators as ops
from oracle import unroll as ur
from oracle import wapg as wp
from oracle.philox import gaussian_matrix
from workloads import phantom


def _setup(n=16, k=3, ell=8, lam=2e-2, seed=4, precond=True):
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.2, 1.0, (k, k))
    h /= h.sum()                           # non-symmetric: catches a flipped kernel
    op = ops.Operator("blur", n, n, kernel=h)
    x_true = phantom(n, 4, seed, "mixed")
    y = op.apply(x_true) + rng.normal(0, 0.01, (n, n))
    prob = wp.Problem(op, y, lam, "tv")
    if precond:
        phi = lambda V: prob.phi(V.reshape(-1, n, n)).reshape(V.shape[0], -1)
        r = ny.nystrom(phi, gaussian_matrix(n * n, ell, seed=seed + 1), 2.0 ** -52)
        P = ny.Precond(r["U"], r["S_hat"])
    else:
        P = ny.Identity()
    alpha = 1.0 / wp.power_lipschitz(prob, P if precond else None)
    return op, y, x_true, prob, P, alpha


def _loss(h, lam, y, x_true, P, alpha, K, J, n):
    op = ops.Operator("blur", n, n, kernel=h)
    xK, _ = ur.forward(op, y, lam, alpha, P, K, J)
    return float(np.mean((xK - x_true) ** 2))


@pytest.mark.parametrize("precond", [True, False])
def test_unrolled_forward_is_algorithm_3(precond):
    op, y, x_true, prob, P, alpha = _setup(precond=precond)
    xK, _ = ur.forward(op, y, prob.lam, alpha, P, 7, 5)
    ref = wp.wapg(prob, alpha, 7, precond=P if precond else None, n_inner=5)["x"]
    assert np.abs(xK - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("precond", [True, False])
def test_gradient_matches_central_differences(precond):
    n, K, J = 16, 6, 5
    op, y, x_true, prob, P, alpha = _setup(n=n, precond=precond)
    loss, dlam, dh = ur.value_and_grad(op, y, prob.lam, alpha, P, K, J, x_true)
    h = op.kernel
    assert loss == pytest.approx(_loss(h, prob.lam, y, x_true, P, alpha, K, J, n), rel=1e-14)
    e = 1e-6 * prob.lam
    fd = (_loss(h, prob.lam + e, y, x_true, P, alpha, K, J, n)
          - _loss(h, prob.lam - e, y, x_true, P, alpha, K, J, n)) / (2 * e)
    assert abs(dlam - fd) <= 1e-6 * abs(fd), (dlam, fd)
    fdh = np.zeros_like(h)
    for a in range(h.shape[0]):
        for b in range(h.shape[1]):
            hp, hm = h.copy(), h.copy()
            hp[a, b] += 1e-6
            hm[a, b] -= 1e-6
            fdh[a, b] = (_loss(hp, prob.lam, y, x_true, P, alpha, K, J, n)
                         - _loss(hm, prob.lam, y, x_true, P, alpha, K, J, n)) / 2e-6
    assert np.linalg.norm(dh - fdh) <= 1e-6 * np.linalg.norm(fdh), (dh, fdh)


def test_gradient_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    n, K, J = 16, 8, 6
    op, y, x_true, prob, P, alpha = _setup(n=n, k=5, seed=9)
    loss, dlam, dh = ur.value_and_grad(op, y, prob.lam, alpha, P, K, J, x_true)

    # independent re-statement of the forward map in torch ops
    U = torch.from_numpy(P.U)
    dinv = torch.from_numpy(1.0 / (1.0 + P.d) - 1.0)

    def pinv(z):
        zf = z.reshape(-1)
        return (zf + U.T @ (dinv * (U @ zf))).reshape(z.shape)   # U is ell x N

    def blur(x, hh):
        kh = hh.shape[0]
        c = (kh - 1) // 2
        out = torch.zeros_like(x)
        for a in range(kh):
            for b in range(kh):
                out = out + hh[a, b] * torch.roll(x, shifts=(-(a - c), -(b - c)), dims=(0, 1))
        return out

    def blur_t(x, hh):
        kh = hh.shape[0]
        c = (kh - 1) // 2
        out = torch.zeros_like(x)
        for a in range(kh):
            for b in range(kh):
                out = out + hh[a, b] * torch.roll(x, shifts=(a - c, b - c), dims=(0, 1))
        return out

    def D(x):
        return torch.stack([x - torch.roll(x, 1, 0), x - torch.roll(x, 1, 1)])

    def Dt(q):
        return (q[0] - torch.roll(q[0], -1, 0)) + (q[1] - torch.roll(q[1], -1, 1))

    hh = torch.from_numpy(op.kernel.copy()).requires_grad_(True)
    lam = torch.tensor(prob.lam, dtype=torch.float64, requires_grad=True)
    yt = torch.from_numpy(y)
    lb = alpha * lam
    x = torch.zeros(n, n, dtype=torch.float64)
    u = x.clone()
    Q = torch.zeros(2, n, n, dtype=torch.float64)
    tp = 1.0
    for _ in range(K):
        s = u - alpha * pinv(blur_t(blur(u, hh) - yt, hh))
        Qp, R, t = Q, Q, 1.0
        for _ in range(J):
            z = R + (1.0 / (8.0 * lb)) * D(s - lb * pinv(Dt(R)))
            Qn = torch.clamp(z, -1.0, 1.0)
            tn = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
            R = Qn + ((t - 1.0) / tn) * (Qn - Qp)
            Qp, t = Qn, tn
        Q = Qp
        xn = s - lb * pinv(Dt(Q))
        tk = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * tp * tp))
        u = xn + ((tp - 1.0) / tk) * (xn - x)
        x, tp = xn, tk
    L = torch.mean((x - torch.from_numpy(x_true)) ** 2)
    L.backward()
    assert float(L.detach()) == pytest.approx(loss, rel=1e-12)
    assert abs(float(lam.grad) - dlam) <= 1e-10 * abs(dlam)
    g = hh.grad.numpy()
    assert np.linalg.norm(g - dh) <= 1e-10 * np.linalg.norm(g)


def test_kernel_grad_closed_form():
    # d<w, h (*) x>/dh[a,b] at the centre tap is <w, x>; a delta image x picks
    # out w at the shifted position
    rng = np.random.default_rng(0)
    w = rng.standard_normal((8, 8))
    x = np.zeros((8, 8))
    x[2, 5] = 1.0
    g = ur.blur_kernel_grad(w, x, (3, 3))
    # x[i + a - 1, j + b - 1] = 1  <=>  (i, j) = (3 - a, 6 - b)
    for a in range(3):
        for b in range(3):
            assert g[a, b] == w[3 - a, 6 - b]
    assert ur.blur_kernel_grad(w, w, (1, 1))[0, 0] == pytest.approx(np.sum(w * w))
