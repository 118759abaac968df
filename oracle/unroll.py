"""Unrolled preconditioned WAPG and its reverse-mode gradient (oracle, float64).

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

The map differentiated is K iterations of Algorithm 3 with the anisotropic TV
regulariser, whose P-metric prox is the dual APG of Sec. III-B run for a fixed
n_inner steps with its dual variable Q warm-started from the previous outer
iteration (exactly what oracle.wapg.wapg computes for reg="tv"):

    r_k  = A u_k - y,   g_k = A^T r_k,   s_k = u_k - alpha P^{-1} g_k
    dual steps j = 0 .. J-1 (R_0 = Q_0 = warm start, t_0 = 1):
        x_j     = s_k - lam_bar P^{-1} L^T R_j
        z_j     = R_j + (1 / (8 lam_bar)) L x_j
        Q_{j+1} = clip(z_j, -1, 1)
        R_{j+1} = Q_{j+1} + beta_j (Q_{j+1} - Q_j),  beta_j = (t_j - 1)/t_{j+1}
    x_{k+1} = s_k - lam_bar P^{-1} L^T Q_J
    u_{k+1} = x_{k+1} + gamma_k (x_{k+1} - x_k)

with lam_bar = alpha lambda, L the periodic backward-difference gradient and
x_0 = u_0 = 0, Q = 0 at k = 0.  The loss is the mean squared error
mean((x_K - x_ref)^2).  The preconditioner P and the step size alpha are held
fixed (they are built once for the starting kernel and are not functions of
the parameters), so the gradient is that of the unrolled map as written.

The reverse pass below is derived by hand, one line per forward assignment
read backwards; clip has derivative 1 strictly inside (-1, 1) and 0 outside.
For the blur A x = h (*) x (correlation form), the derivative of <w, A x> with
respect to the tap h[a, b] is sum_{i,j} w[i,j] x[i+a-c, j+b-c]
(`blur_kernel_grad`).
"""
from __future__ import annotations

import math

import numpy as np

from . import operators as ops


def blur_kernel_grad(w: np.ndarray, x: np.ndarray, kshape) -> np.ndarray:
    """d <w, h (*) x> / dh for the periodic correlation blur (Sec. IV deblurring model)."""
    kh, kw = kshape
    ch, cw = (kh - 1) // 2, (kw - 1) // 2
    out = np.zeros((kh, kw))
    for a in range(kh):
        for b in range(kw):
            out[a, b] = float(np.sum(w * np.roll(x, shift=(-(a - ch), -(b - cw)), axis=(-2, -1))))
    return out


def _momentum_coeffs(count: int):
    """t_k and (t_{k-1} - 1)/t_k for k = 1 .. count, t_0 = 1 (Alg. 3)."""
    t_prev, out = 1.0, []
    for _ in range(count):
        t = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t_prev * t_prev))
        out.append((t_prev - 1.0) / t)
        t_prev = t
    return out


def forward(op, y, lam: float, alpha: float, precond, K: int, n_inner: int, record: bool = False):
    """K unrolled iterations; returns (x_K, tape).  tape (if record) holds per
    outer iteration u_k, r_k, Q_0 and the dual iterates z_j."""
    shape = (op.n1, op.n2)
    lam_bar = alpha * lam
    step = 1.0 / (8.0 * lam_bar)
    gammas = _momentum_coeffs(K)
    betas = _momentum_coeffs(n_inner)
    x = np.zeros(shape)
    u = np.zeros(shape)
    Q = np.zeros((2,) + shape)
    tape = []
    for k in range(K):
        r = op.apply(u) - y
        s = u - alpha * precond.inverse(op.adjoint(r))
        Q0 = Q
        Q_prev, R = Q, Q
        zs = []
        for j in range(n_inner):
            xj = s - lam_bar * precond.inverse(ops.grad_adjoint(R))
            z = R + step * ops.grad(xj)
            Qn = np.clip(z, -1.0, 1.0)
            R = Qn + betas[j] * (Qn - Q_prev)
            Q_prev = Qn
            zs.append(z)
        Q = Q_prev
        x_new = s - lam_bar * precond.inverse(ops.grad_adjoint(Q))
        u_new = x_new + gammas[k] * (x_new - x)
        if record:
            tape.append(dict(u=u, r=r, Q0=Q0, zs=zs))
        x, u = x_new, u_new
    return x, tape


def value_and_grad(op, y, lam: float, alpha: float, precond, K: int, n_inner: int, x_ref,
                   kernel_grad: bool = True):
    """(loss, d loss / d lambda, d loss / d h) for loss = mean((x_K - x_ref)^2).
    d/dh is returned only for the blur operator (None otherwise)."""
    xK, tape = forward(op, y, lam, alpha, precond, K, n_inner, record=True)
    N = xK.size
    loss = float(np.mean((xK - x_ref) ** 2))
    lam_bar = alpha * lam
    step = 1.0 / (8.0 * lam_bar)
    gammas = _momentum_coeffs(K)
    betas = _momentum_coeffs(n_inner)
    want_h = kernel_grad and op.kind == "blur"
    dh = np.zeros(op.kernel.shape) if want_h else None
    dlam_bar = 0.0
    xbar = 2.0 * (xK - x_ref) / N          # adjoint of x_{k+1}, partial
    ubar_next = np.zeros_like(xK)           # adjoint of u_{k+1}
    Qbar_next = np.zeros((2,) + xK.shape)   # adjoint of the Q handed to iteration k+1
    for k in reversed(range(K)):
        rec = tape[k]
        g = gammas[k]
        # u_{k+1} = (1 + g) x_{k+1} - g x_k
        xbar_new = xbar + (1.0 + g) * ubar_next
        xbar_old = -g * ubar_next
        # recover the dual iterates: Q_0 given, Q_{j+1} = clip(z_j)
        Qs = [rec["Q0"]] + [np.clip(z, -1.0, 1.0) for z in rec["zs"]]
        Rs = [Qs[0]] + [Qs[j + 1] + betas[j] * (Qs[j + 1] - Qs[j]) for j in range(n_inner)]
        # x_{k+1} = s - lam_bar P^{-1} L^T Q_J
        sbar = xbar_new.copy()
        w = precond.inverse(xbar_new)
        Lw = ops.grad(w)
        Qbar = Qbar_next - lam_bar * Lw
        dlam_bar -= float(np.sum(Lw * Qs[n_inner]))
        Rbar = np.zeros_like(Qbar)
        for j in reversed(range(n_inner)):
            b = betas[j]
            # R_{j+1} = (1 + b) Q_{j+1} - b Q_j
            Qbar_j1 = Qbar + (1.0 + b) * Rbar
            Qbar = -b * Rbar
            # Q_{j+1} = clip(z_j)
            z = rec["zs"][j]
            zbar = Qbar_j1 * (np.abs(z) < 1.0)
            # z_j = R_j + step L x_j
            Lx = (z - Rs[j]) / step
            Rbar = zbar.copy()
            dlam_bar += (-step / lam_bar) * float(np.sum(zbar * Lx))
            xbar_j = step * ops.grad_adjoint(zbar)
            # x_j = s - lam_bar P^{-1} L^T R_j
            sbar += xbar_j
            w = precond.inverse(xbar_j)
            Lw = ops.grad(w)
            Rbar -= lam_bar * Lw
            dlam_bar -= float(np.sum(Lw * Rs[j]))
        # R_0 = Q_0 (the warm start)
        Qbar_next = Qbar + Rbar
        # s = u - alpha P^{-1} g,  g = A^T r,  r = A u - y
        ubar = sbar.copy()
        gbar = -alpha * precond.inverse(sbar)
        rbar = op.apply(gbar)
        ubar += op.adjoint(rbar)
        if want_h:
            dh += blur_kernel_grad(rec["r"], gbar, op.kernel.shape)    # the A of A^T r
            dh += blur_kernel_grad(rbar, rec["u"], op.kernel.shape)    # the A of A u
        ubar_next = ubar
        xbar = xbar_old
    return loss, alpha * dlam_bar, dh
