"""Weighted proximal mappings in the P-metric (oracle side, float64).

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

* prox_wavelet: Theorem 1 (Becker et al.) with D = I and W = I + Ubar Ubar^T:
      prox^W_{tau||.||_1}(s) = T_tau(s - Ubar gamma*),
      gamma* solves F(gamma) = Ubar^T (s - T_tau(s - Ubar gamma)) + gamma = 0,
  with T_tau the soft threshold.  F is solved by semi-smooth Newton (the paper
  names the method but gives no details), read as: generalised Jacobian
  J = I + Ubar^T diag(1[|z| > tau]) Ubar at z = s - Ubar gamma (strict
  inequality), plain Newton step, step halved (at most 10 times) while ||F||
  does not decrease, stop when ||F|| <= tol (1 + ||Ubar^T s||) or after 50
  steps.
* prox_dual: the dual scheme of Sec. III-B for g(x) = ||L x||_{1,phi} with
  C = R^N: the dual objective ||s - lb P^{-1} L^T Q||_P^2 over the unit ball
  B of the dual mixed norm has gradient -2 lb L x(Q), x(Q) = s - lb P^{-1} L^T Q,
  and Lipschitz constant 2 lb^2 ||L||^2 (sigma_min(P) = 1).  It is minimised
  by APG (FISTA) for a fixed number of steps n_inner, warm-started from Q0:
      x   = s - lb P^{-1} L^T R_k
      Q_k = Proj_B(R_k + L x / (lb ||L||^2))
      t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
      R_{k+1} = Q_k + ((t_k - 1)/t_{k+1}) (Q_k - Q_{k-1})
  and returns x(Q_n) and Q_n.  The dual ball is the unit ball of the mixed
  norm l_{inf,psi}, 1/phi + 1/psi = 1 (Eqs. dualMixedNormRep and
  mixedUnitNormBall); its projection acts on each group (pixel) alone:
    - anisotropic TV (phi = 1, psi = inf): clip every component to [-1, 1];
    - isotropic TV (phi = 2, psi = 2): scale each pixel's pair to Euclidean
      norm <= 1;
    - Hessian Schatten-1 (HS_1: phi = 1 on the singular values of the 2x2
      Hessian, dual ball = spectral norm <= 1): clip the eigenvalues;
    - Hessian Schatten-2 (HS_2, Frobenius, self-dual): scale each symmetric
      block to Frobenius norm <= 1 (the cross term counted twice, as in the
      inner product q11 v11 + 2 q12 v12 + q22 v22);
    - Hessian Schatten-inf (HS_inf, spectral norm; dual ball = Schatten-1
      norm <= 1): project the eigenvalue pair onto the l1 unit ball.
  (Appendix A gives the groups; the Hessian variants are the HS_1, HS_2 and
  HS_inf of the supplementary CT experiments.)
"""
from __future__ import annotations

import numpy as np

from . import operators as ops


def soft_threshold(z, tau):
    return np.sign(z) * np.maximum(np.abs(z) - tau, 0.0)


def prox_wavelet(s: np.ndarray, Ubar: np.ndarray | None, tau: float,
                 gamma0: np.ndarray | None = None, tol: float = 1e-12, max_iter: int = 50):
    """Theorem 1 prox.  s: (N,), Ubar: (r, N) rows or None (P = I).

    Returns (x, gamma, n_newton, converged).
    """
    s = np.asarray(s, dtype=np.float64).reshape(-1)
    if Ubar is None or Ubar.shape[0] == 0:
        return soft_threshold(s, tau), None, 0, True
    Ub = np.asarray(Ubar, dtype=np.float64)
    r = Ub.shape[0]
    g = np.zeros(r) if gamma0 is None else np.array(gamma0, dtype=np.float64)
    scale = 1.0 + np.linalg.norm(Ub @ s)

    def F(gam):
        z = s - gam @ Ub
        return Ub @ (s - soft_threshold(z, tau)) + gam, z

    Fg, z = F(g)
    nF = np.linalg.norm(Fg)
    it = 0
    while nF > tol * scale and it < max_iter:
        mask = (np.abs(z) > tau).astype(np.float64)
        J = np.eye(r) + (Ub * mask[None, :]) @ Ub.T
        step = -np.linalg.solve(J, Fg)
        a = 1.0
        for _ in range(11):
            g_new = g + a * step
            F_new, z_new = F(g_new)
            n_new = np.linalg.norm(F_new)
            if n_new < nF:
                break
            a *= 0.5
        g, Fg, z, nF = g_new, F_new, z_new, n_new
        it += 1
    x = soft_threshold(s - g @ Ub, tau)
    return x, g, it, bool(nF <= tol * scale)


def proj_box(q):
    return np.clip(q, -1.0, 1.0)


def proj_spectral_2x2(q):
    """q: (..., 3, n1, n2) holding (a, b, c) of [[a, b], [b, c]] per pixel."""
    a, b, c = q[..., 0, :, :], q[..., 1, :, :], q[..., 2, :, :]
    m = 0.5 * (a + c)
    h = 0.5 * (a - c)
    r = np.sqrt(h * h + b * b)
    l1 = np.clip(m + r, -1.0, 1.0)
    l2 = np.clip(m - r, -1.0, 1.0)
    mp = 0.5 * (l1 + l2)
    dp = 0.5 * (l1 - l2)
    safe = np.where(r > 0.0, r, 1.0)
    cos2, sin2 = np.where(r > 0.0, h / safe, 1.0), np.where(r > 0.0, b / safe, 0.0)
    return np.stack([mp + dp * cos2, dp * sin2, mp - dp * cos2], axis=-3)


def proj_l2_pairs(q):
    """q: (..., 2, n1, n2); each pixel's (q1, q2) scaled to Euclidean norm <= 1."""
    nrm = np.sqrt(q[..., 0, :, :] ** 2 + q[..., 1, :, :] ** 2)
    return q / np.maximum(1.0, nrm)[..., None, :, :]


def proj_frobenius_2x2(q):
    """q: (..., 3, n1, n2) holding (a, b, c) of [[a, b], [b, c]]; each block
    scaled to Frobenius norm sqrt(a^2 + 2 b^2 + c^2) <= 1."""
    a, b, c = q[..., 0, :, :], q[..., 1, :, :], q[..., 2, :, :]
    nrm = np.sqrt(a * a + 2.0 * b * b + c * c)
    return q / np.maximum(1.0, nrm)[..., None, :, :]


def proj_l1_ball_2(l1, l2):
    """Euclidean projection of the pairs (l1, l2) onto |l1| + |l2| <= 1:
    soft-thresholding by the theta that brings the sum of magnitudes to 1."""
    a1, a2 = np.abs(l1), np.abs(l2)
    big, small = np.maximum(a1, a2), np.minimum(a1, a2)
    theta = np.where(big - small >= 1.0, big - 1.0, 0.5 * (big + small - 1.0))
    theta = np.where(a1 + a2 <= 1.0, 0.0, theta)
    return np.sign(l1) * np.maximum(a1 - theta, 0.0), np.sign(l2) * np.maximum(a2 - theta, 0.0)


def proj_nuclear_2x2(q):
    """q: (..., 3, n1, n2) as in proj_spectral_2x2; each block projected onto
    the Schatten-1 (nuclear) unit ball: its eigenvalue pair onto the l1 ball."""
    a, b, c = q[..., 0, :, :], q[..., 1, :, :], q[..., 2, :, :]
    m = 0.5 * (a + c)
    h = 0.5 * (a - c)
    r = np.sqrt(h * h + b * b)
    l1, l2 = proj_l1_ball_2(m + r, m - r)
    mp = 0.5 * (l1 + l2)
    dp = 0.5 * (l1 - l2)
    safe = np.where(r > 0.0, r, 1.0)
    cos2, sin2 = np.where(r > 0.0, h / safe, 1.0), np.where(r > 0.0, b / safe, 0.0)
    return np.stack([mp + dp * cos2, dp * sin2, mp - dp * cos2], axis=-3)


REGULARISERS = {
    # name: (L, L^T, ||L||^2, projection onto the dual unit ball)
    "tv": (ops.grad, ops.grad_adjoint, 8.0, proj_box),
    "isotv": (ops.grad, ops.grad_adjoint, 8.0, proj_l2_pairs),
    "hs": (ops.hess, ops.hess_adjoint, 32.0, proj_spectral_2x2),
    "hs2": (ops.hess, ops.hess_adjoint, 32.0, proj_frobenius_2x2),
    "hsinf": (ops.hess, ops.hess_adjoint, 32.0, proj_nuclear_2x2),
}
DUAL_COMPONENTS = {"tv": 2, "isotv": 2, "hs": 3, "hs2": 3, "hsinf": 3}


def prox_dual(s: np.ndarray, reg: str, lam_bar: float, precond, n_inner: int,
              Q0: np.ndarray | None = None):
    """Dual APG for prox^P_{lam_bar ||L.||_{1,phi}}(s).  s: (n1, n2).

    precond: object with .inverse(z) (oracle.nystrom.Precond or Identity).
    Returns (x, Q).
    """
    L, Lt, normL2, proj = REGULARISERS[reg]
    s = np.asarray(s, dtype=np.float64)
    G = DUAL_COMPONENTS[reg]
    Q_prev = np.zeros((G,) + s.shape) if Q0 is None else np.array(Q0, dtype=np.float64)
    R = Q_prev.copy()
    t = 1.0
    step = 1.0 / (lam_bar * normL2)
    for _ in range(n_inner):
        x = s - lam_bar * precond.inverse(Lt(R))
        Q = proj(R + step * L(x))
        t_next = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        R = Q + ((t - 1.0) / t_next) * (Q - Q_prev)
        Q_prev, t = Q, t_next
    x = s - lam_bar * precond.inverse(Lt(Q_prev))
    return x, Q_prev


def reg_value(x: np.ndarray, reg: str) -> float:
    """g(x) = ||L x||_{1,phi}: anisotropic or isotropic TV, Hessian Schatten-1, -2
    or -inf, or l1 (wavelet coefficients)."""
    if reg == "tv":
        return float(np.abs(ops.grad(x)).sum())
    if reg == "isotv":
        g = ops.grad(x)
        return float(np.sqrt(g[0] ** 2 + g[1] ** 2).sum())
    if reg in ("hs", "hs2", "hsinf"):
        v = ops.hess(x)
        a, b, c = v[0], v[1], v[2]
        if reg == "hs2":
            return float(np.sqrt(a * a + 2.0 * b * b + c * c).sum())
        m = 0.5 * (a + c)
        r = np.sqrt((0.5 * (a - c)) ** 2 + b * b)
        if reg == "hsinf":
            return float((np.abs(m) + r).sum())
        return float((np.abs(m + r) + np.abs(m - r)).sum())
    if reg == "wavelet":
        return float(np.abs(x).sum())
    raise ValueError(reg)
