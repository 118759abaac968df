"""Randomized Nystrom approximation and preconditioner (oracle side, float64).

TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

Follows Algorithm 1 step by step, in the paper's notation, with columns of
Omega, Y, U stored as rows of (ell, N) arrays (each probe column is an image):
  1. Omega ~ N(0,1)^{N x K}            (oracle.philox.gaussian_matrix)
  2. Y = Phi Omega                      (Phi applied column by column)
  3. v = eps ||Omega||_F
  4. Y_v = Y + v Omega
  5. C = chol(Omega^T Y_v)              (lower, C C^T = sym(Omega^T Y_v))
  6. B = Y_v C^{-T}
  7. [U, S, ~] = SVD(B)                 (thin, descending)
  8. S_hat = max(0, S^2 - v)
Readings of points the paper leaves open:
  * the core Omega^T Y_v is symmetrised as (M + M^T)/2 before the Cholesky;
  * if the Cholesky fails, v is multiplied by 10 and steps 4-5 repeated, at most
    8 times.
The preconditioner is Eq. (RYPreconditioner) rewritten as P = I + Ubar Ubar^T
(Sec. III-B):  with s' = sqrt(s_K) when the square-root heuristic is on (the
paper's choice for WAPG) and s' = s_K otherwise,
    d_i = max(0, (s_i + mu)/(s' + mu) - 1),   Ubar = U diag(sqrt(d)),
    P z    = z + U diag(d) U^T z,
    P^{-1} z = z + U diag(1/(1+d) - 1) U^T z.
Without the clamp and the heuristic, d_K = 0 and these are exactly the two
lines of Eq. (RYPreconditioner); the clamp keeps P >= I when sqrt(s_K) > s_i.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


class NotSPD(RuntimeError):
    pass


class Degenerate(RuntimeError):
    pass


def nystrom(phi, omega: np.ndarray, eps: float, max_retries: int = 8):
    """Algorithm 1.  phi maps an (ell, N) stack of vectors to Phi applied to each.

    Returns dict(U=(ell, N), S_hat=(ell,), v=float, retries=int, Y=(ell, N)).
    """
    omega = np.asarray(omega, dtype=np.float64)
    Y = np.asarray(phi(omega), dtype=np.float64)                     # step 2
    v = eps * np.linalg.norm(omega)                                   # step 3
    for retries in range(max_retries + 1):
        Yv = Y + v * omega                                            # step 4
        M = omega @ Yv.T                                              # Omega^T Y_v
        M = 0.5 * (M + M.T)
        try:
            C = np.linalg.cholesky(M)                                 # step 5
            break
        except np.linalg.LinAlgError:
            v *= 10.0
    else:
        raise NotSPD("Cholesky of the shifted core failed after retries")
    # step 6: B = Y_v C^{-T}  <=>  C B^T = Y_v^T
    Bt = scipy.linalg.solve_triangular(C, Yv, lower=True)             # (ell, N) = B^T
    U, S, _ = np.linalg.svd(Bt.T, full_matrices=False)                # step 7
    S_hat = np.maximum(0.0, S * S - v)                                # step 8
    return dict(U=U.T.copy(), S_hat=S_hat, v=v, retries=retries, Y=Y)


def precond_weights(S_hat: np.ndarray, mu: float = 0.0, sqrt_shift: bool = True):
    """d_i of P = I + U diag(d) U^T (clamped at 0)."""
    s_k = float(S_hat[-1])
    s_ref = np.sqrt(s_k) if sqrt_shift else s_k
    if not (s_ref + mu > 0.0):
        raise Degenerate("s_K + mu must be positive")
    return np.maximum(0.0, (S_hat + mu) / (s_ref + mu) - 1.0)


class Precond:
    """P = I + U diag(d) U^T and its inverse, U stored as (ell, N) rows."""

    def __init__(self, U: np.ndarray, S_hat: np.ndarray, mu: float = 0.0, sqrt_shift: bool = True):
        self.U = np.asarray(U, dtype=np.float64)
        self.d = precond_weights(np.asarray(S_hat, dtype=np.float64), mu, sqrt_shift)

    @property
    def Ubar(self) -> np.ndarray:
        return self.U * np.sqrt(self.d)[:, None]

    def _low_rank(self, z, diag):
        N = self.U.shape[1]
        flat = z if z.shape[-1] == N else z.reshape(z.shape[:-2] + (N,))
        w = flat @ self.U.T                      # U^T z
        return (flat + (w * diag) @ self.U).reshape(z.shape)

    def apply(self, z):
        return self._low_rank(np.asarray(z, dtype=np.float64), self.d)

    def inverse(self, z):
        return self._low_rank(np.asarray(z, dtype=np.float64), 1.0 / (1.0 + self.d) - 1.0)


class Identity:
    """P = I (plain APG)."""
    U = None

    def apply(self, z):
        return np.asarray(z, dtype=np.float64)

    def inverse(self, z):
        return np.asarray(z, dtype=np.float64)
