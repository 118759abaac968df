"""Weighted accelerated proximal gradient (Algorithm 3) and helpers (oracle, float64).

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

Algorithm 3, for k = 1 .. MaxIter:
    x^{k+1} = prox^P_{(alpha lambda) g}(u^k - alpha P^{-1} grad f(u^k))
    t^k     = (1 + sqrt(1 + 4 (t^{k-1})^2)) / 2
    u^{k+1} = x^{k+1} + ((t^{k-1} - 1)/t^k) (x^{k+1} - x^k)
with t^0 = 1; P = I gives plain APG.  Readings: x^1 = u^1 = 0; C = R^N.
Data terms: f(x) = 1/2 ||A x - y||^2 (Eq. 3 with p = 2), or the Huber loss
sum h_delta((A x - y)_m) with h_delta(r) = r^2/2 for |r| <= delta and
delta |r| - delta^2/2 otherwise, whose gradient is A^T clip(A x - y, -delta, delta).
For the wavelet regulariser the problem is posed in the coefficients
xbar = W x (Sec. III-B, invertible L): f(xbar) = 1/2 ||A W^T xbar - y||^2 and
g(xbar) = ||xbar||_1, so Phi = W A^T A W^T.
The step size is alpha = 1/L_f^P; L_f^P is estimated as 1.02 times the
largest eigenvalue of P^{-1} Phi found by 50 power-iteration steps.
"""
from __future__ import annotations

import math

import numpy as np

from . import operators as ops
from . import prox as px
from .nystrom import Identity


class Problem:
    """min_x f(x) + lambda g(x) for one operator, data y and regulariser."""

    def __init__(self, op: ops.Operator, y: np.ndarray, lam: float, reg: str,
                 fit: str = "l2", huber_delta: float = 0.0, haar_levels: int = 3, wavelet: str = "haar"):
        self.op, self.y, self.lam, self.reg = op, np.asarray(y, dtype=np.float64), lam, reg
        self.fit, self.delta, self.levels, self.wavelet = fit, huber_delta, haar_levels, wavelet
        self.shape = (op.n1, op.n2)

    # variable <-> image
    def _w(self, x):
        if self.wavelet == "haar":
            return ops.haar_forward(x, self.levels)
        return ops.wavelet_forward(x, self.levels, self.wavelet)

    def _wt(self, c):
        if self.wavelet == "haar":
            return ops.haar_adjoint(c, self.levels)
        return ops.wavelet_adjoint(c, self.levels, self.wavelet)

    def to_image(self, v):
        return self._wt(v) if self.reg == "wavelet" else v

    def phi(self, v):
        """Phi = A^T A (or W A^T A W^T) applied to a stack of variables (..., n1, n2)."""
        if self.reg == "wavelet":
            return self._w(self.op.normal(self._wt(v)))
        return self.op.normal(v)

    def grad_f(self, v):
        r = self.op.apply(self.to_image(v)) - self.y
        if self.fit == "huber":
            r = np.clip(r, -self.delta, self.delta)
        g = self.op.adjoint(r)
        return self._w(g) if self.reg == "wavelet" else g

    def objective(self, v) -> float:
        r = self.op.apply(self.to_image(v)) - self.y
        if self.fit == "huber":
            a = np.abs(r)
            f = np.where(a <= self.delta, 0.5 * r * r, self.delta * a - 0.5 * self.delta ** 2).sum()
        else:
            f = 0.5 * float(np.sum(r * r))
        return float(f) + self.lam * px.reg_value(v, self.reg)


def power_lipschitz(prob: Problem, precond=None, iters: int = 50, seed: int = 7,
                    safety: float = 1.02) -> float:
    """safety * largest eigenvalue of P^{-1} Phi by power iteration."""
    P = precond if precond is not None else Identity()
    z = np.random.default_rng(seed).standard_normal(prob.shape)
    z /= np.linalg.norm(z)
    lam = 0.0
    for _ in range(iters):
        w = P.inverse(prob.phi(z))
        lam = float(np.linalg.norm(w))
        z = w / lam
    return safety * lam


def wapg(prob: Problem, alpha: float, iters: int, precond=None, n_inner: int = 20,
         x1: np.ndarray | None = None, sqrt_gamma_warm: bool = True, callback=None,
         momentum: bool = True):
    """Algorithm 3.  Returns dict(x, Q, gamma, xs) with x the final variable.

    momentum=False gives the unaccelerated proximal gradient (t fixed at 1).
    callback(k, x) is called after each iteration.
    """
    P = precond if precond is not None else Identity()
    Ubar = None if (precond is None or getattr(precond, "U", None) is None) else precond.Ubar
    x_prev = np.zeros(prob.shape) if x1 is None else np.array(x1, dtype=np.float64)
    u = x_prev.copy()
    t_prev = 1.0
    Q = None
    gamma = None
    tau = alpha * prob.lam
    for k in range(1, iters + 1):
        s = u - alpha * P.inverse(prob.grad_f(u))
        if prob.reg == "wavelet":
            xf, gamma, _, _ = px.prox_wavelet(s.reshape(-1), Ubar, tau,
                                              gamma if sqrt_gamma_warm else None)
            x_new = xf.reshape(prob.shape)
        else:
            x_new, Q = px.prox_dual(s, prob.reg, tau, P, n_inner, Q)
        if momentum:
            t = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t_prev * t_prev))
            u = x_new + ((t_prev - 1.0) / t) * (x_new - x_prev)
            t_prev = t
        else:
            u = x_new
        x_prev = x_new
        if callback is not None:
            callback(k, x_new)
    return dict(x=x_prev, Q=Q, gamma=gamma)
