"""Pins for the oracle's IRM with (P)CG (Algorithm 2, Eqs. halfQuad,
v:z:updating, WfWg:IRM, lplq:sub:updateX:linearEq).

* the half-quadratic constants: |r|^p equals the minimum over beta of
  beta r^2 + 1/(b_p beta^{a_p}), attained at beta* = (p/2)|r|^{p-2};
* with p = q = 2 every weight is 1 and one IRM step is the dense solve of
  (A^T A + lambda L^T L) x = A^T y;
* PCG with the exact inverse as preconditioner converges in one step, plain
  CG reaches the residual tolerance, and both agree with a dense solve;
* every IRM step decreases the smoothed objective (a majorise-minimise step,
  also with inexact CG started from the previous iterate);
* the on-the-fly Nystrom preconditioner cuts the CG iterations.
"""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import irm as ir
from oracle import operators as ops
from workloads import gaussian_kernel, phantom


@pytest.mark.parametrize("p", [0.5, 0.8, 1.0, 1.5])
def test_half_quadratic_representation(p):
    a, b = ir.half_quadratic_constants(p)
    for r in (0.03, 0.7, 2.5):
        f = lambda beta: beta * r * r + 1.0 / (b * beta ** a)
        beta_star = 0.5 * p * abs(r) ** (p - 2.0)
        assert f(beta_star) == pytest.approx(abs(r) ** p, rel=1e-12)
        res = minimize_scalar(lambda lb: f(np.exp(lb)), bounds=(-20, 20), method="bounded",
                              options={"xatol": 1e-12})
        assert res.fun == pytest.approx(abs(r) ** p, rel=1e-8)
        assert np.exp(res.x) == pytest.approx(beta_star, rel=1e-4)


def _problem(n=10, k=5, seed=0, impulsive=True):
    rng = np.random.default_rng(seed)
    op = ops.Operator("blur", n, n, kernel=gaussian_kernel(k, 1.2))
    x_true = phantom(n, 4, seed, "mixed")
    y = op.apply(x_true) + rng.normal(0, 0.01, (n, n))
    if impulsive:
        m = rng.uniform(size=(n, n))
        y = np.where(m < 0.05, 1.0, np.where(m > 0.95, 0.0, y))
    return op, y


def _dense(apply, n):
    E = np.eye(n * n)
    return np.stack([apply(E[i].reshape(n, n)).reshape(-1) for i in range(n * n)], axis=1)


def test_quadratic_case_is_one_linear_solve():
    n, lam = 8, 0.05
    op, y = _problem(n, 3, 1, impulsive=False)
    x, hist = ir.irm(op, y, lam, 2.0, 2.0, 1e-3, outer=1, cg_tol=1e-13, cg_max=1000)
    H = _dense(lambda v: op.adjoint(op.apply(v)) + lam * ops.grad_adjoint(ops.grad(v)), n)
    x_ref = np.linalg.solve(H, op.adjoint(y).reshape(-1)).reshape(n, n)
    assert np.abs(x - x_ref).max() <= 1e-10 * np.abs(x_ref).max()


def test_pcg_exact_preconditioner_and_plain_cg():
    n, lam = 8, 0.03
    op, y = _problem(n, 3, 2)
    x0 = np.zeros((n, n))
    wf = ir.weight(op.apply(x0) - y, 1.0, 1e-4)
    wg = ir.weight(ops.grad(x0 + 0.1 * y), 1.0, 1e-4)
    W = ir.Weighted(op, wf, wg, lam)
    H = _dense(W.apply, n)
    assert np.allclose(H, H.T, atol=1e-12)                      # SPD system
    b = op.adjoint(wf * y)
    x_ref = np.linalg.solve(H, b.reshape(-1)).reshape(n, n)
    Hinv = np.linalg.inv(H)
    x1, it1, res1 = ir.pcg(W.apply, b, x0, 1e-10, 50, lambda v: (Hinv @ v.reshape(-1)).reshape(n, n))
    assert it1 == 1 and res1 <= 1e-10
    x2, it2, res2 = ir.pcg(W.apply, b, x0, 1e-10, 2000)
    assert res2 <= 1e-10 and it2 > 5
    for x in (x1, x2):
        assert np.abs(x - x_ref).max() <= 1e-8 * np.abs(x_ref).max()


@pytest.mark.parametrize("p,q,ell", [(1.0, 1.0, 0), (0.8, 1.0, 12), (1.0, 0.5, 12)])
def test_irm_decreases_the_smoothed_objective(p, q, ell):
    op, y = _problem(12, 5, 3)
    lam, eps = 0.02, 1e-4
    F0 = ir.smoothed_objective(op, y, np.zeros((12, 12)), lam, p, q, eps)
    x, hist = ir.irm(op, y, lam, p, q, eps, outer=5, ell=ell, seed=5, cg_tol=1e-3, cg_max=300)
    F = [F0] + [h["objective"] for h in hist]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(F, F[1:])), F


def test_nystrom_preconditioner_cuts_cg_iterations():
    op, y = _problem(16, 7, 4)
    lam, eps = 0.02, 1e-4
    _, h0 = ir.irm(op, y, lam, 1.0, 1.0, eps, outer=2, ell=0, cg_tol=1e-6, cg_max=2000)
    _, h1 = ir.irm(op, y, lam, 1.0, 1.0, eps, outer=2, ell=40, seed=9, cg_tol=1e-6, cg_max=2000)
    for a, b in zip(h0, h1):
        assert b["residual"] <= 1e-6 and a["residual"] <= 1e-6
        assert b["cg_iters"] < a["cg_iters"], (h0, h1)
