"""Iteratively reweighted minimisation with preconditioned CG (oracle side,
float64) for the l_p - l_q problem of Eq. lplqReg.

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

The problem, componentwise (Eq. lplq:componentwise), with L the first
differences (two components per pixel, each its own element):
    min_x (1/p) sum_m |(A x - y)_m|^p + (lambda/q) sum_l sum_zeta |(L x)_l^zeta|^q .
Half-quadratic form (Eq. halfQuad): |r|^p = min_{beta > 0} beta r^2 +
1/(b_p beta^{a_p}), a_p = p/(2-p), b_p = 2^{2/(2-p)} / ((2-p) p^{p/(2-p)}),
attained at beta* = (p/2) |r|^{p-2} (Eq. halfQuadMin); at r = 0 the paper
uses |r|_eps = sqrt(r^2 + eps).  Algorithm 2 alternates
    v^k = (p/2) |A x^{k-1} - y|_eps^{p-2},  z^k = (q/2) |L x^{k-1}|_eps^{q-2}
(Eq. v:z:updating), W_f = diag((2/p) v^k), W_g = diag((2/q) z^k)
(Eq. WfWg:IRM), and x^k solves (Eq. lplq:sub:updateX:linearEq)
    Phi_k x = A^T W_f y,   Phi_k = A^T W_f A + lambda L^T W_g L,
by CG, preconditioned with the Nystrom preconditioner of Phi_k built on the
fly (Algorithm 1 on a fresh sketch every outer iteration, Eq.
RYPreconditioner with mu = 0).  Readings: eps enters every weight (also at
r != 0); the outer iteration k draws Omega with seed + k; CG starts from
x^{k-1} and stops when the recursively updated residual satisfies
||r|| <= tol ||b||; the preconditioner uses s_K itself (the square-root
heuristic is stated for WAPG).
"""
from __future__ import annotations

import numpy as np

from . import operators as ops
from .nystrom import Precond, nystrom
from .philox import gaussian_matrix


def half_quadratic_constants(p: float):
    """(a_p, b_p) of Eq. halfQuad."""
    a = p / (2.0 - p)
    b = 2.0 ** (2.0 / (2.0 - p)) / ((2.0 - p) * p ** (p / (2.0 - p)))
    return a, b


def weight(r: np.ndarray, p: float, eps: float) -> np.ndarray:
    """(2/p) v with v = (p/2) |r|_eps^{p-2}: the diagonal of W_f (or W_g)."""
    return (r * r + eps) ** (0.5 * (p - 2.0))


def smoothed_objective(op, y, x, lam, p, q, eps) -> float:
    """(1/p) sum |Ax - y|_eps^p + (lambda/q) sum |L x|_eps^q, which every IRM
    step decreases (a majorise-minimise step)."""
    r = op.apply(x) - y
    g = ops.grad(x)
    return float(((r * r + eps) ** (0.5 * p)).sum() / p + lam * ((g * g + eps) ** (0.5 * q)).sum() / q)


class Weighted:
    """Phi_k = A^T W_f A + lambda L^T W_g L, matrix-free."""

    def __init__(self, op, wf, wg, lam):
        self.op, self.wf, self.wg, self.lam = op, wf, wg, lam

    def apply(self, x):
        x = np.asarray(x, dtype=np.float64)
        return self.op.adjoint(self.wf * self.op.apply(x)) + self.lam * ops.grad_adjoint(self.wg * ops.grad(x))


def pcg(apply, b, x0, tol, maxit, pinv=None):
    """Preconditioned conjugate gradients for apply(x) = b from x0.  Returns
    (x, iterations, ||r|| / ||b||)."""
    pinv = pinv if pinv is not None else (lambda v: v)
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - apply(x)
    nb = np.linalg.norm(b)
    if np.linalg.norm(r) <= tol * nb:
        return x, 0, np.linalg.norm(r) / nb
    z = pinv(r)
    d = z.copy()
    rz = float(np.sum(r * z))
    it = 0
    while it < maxit:
        it += 1
        q = apply(d)
        alpha = rz / float(np.sum(d * q))
        x = x + alpha * d
        r = r - alpha * q
        if np.linalg.norm(r) <= tol * nb:
            break
        z = pinv(r)
        rz_new = float(np.sum(r * z))
        d = z + (rz_new / rz) * d
        rz = rz_new
    return x, it, np.linalg.norm(r) / nb


def irm(op, y, lam, p, q, eps, outer, ell=0, seed=0, eps_mach=2.0 ** -52, cg_tol=1e-6, cg_max=500, x0=None):
    """Algorithm 2 with (P)CG for the x-step.  Returns (x, history) with one
    dict per outer iteration: CG iterations, relative change of x, and the
    smoothed objective after the step."""
    n1, n2 = op.n1, op.n2
    N = n1 * n2
    x = np.zeros((n1, n2)) if x0 is None else np.array(x0, dtype=np.float64)
    hist = []
    for k in range(outer):
        wf = weight(op.apply(x) - y, p, eps)
        wg = weight(ops.grad(x), q, eps)
        W = Weighted(op, wf, wg, lam)
        b = op.adjoint(wf * y)
        pinv = None
        if ell:
            phi = lambda V: np.stack([W.apply(v.reshape(n1, n2)).reshape(-1) for v in V])
            res = nystrom(phi, gaussian_matrix(N, ell, seed + k), eps_mach)
            P = Precond(res["U"], res["S_hat"], 0.0, False)
            pinv = lambda v: P.inverse(v.reshape(-1)).reshape(n1, n2)
        x_new, it, res_rel = pcg(W.apply, b, x, cg_tol, cg_max, pinv)
        rel = float(np.linalg.norm(x_new - x) / max(np.linalg.norm(x_new), 1e-300))
        x = x_new
        hist.append(dict(cg_iters=it, residual=res_rel, rel_change=rel,
                         objective=smoothed_objective(op, y, x, lam, p, q, eps)))
    return x, hist
