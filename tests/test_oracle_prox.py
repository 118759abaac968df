"""Pins for the oracle's weighted proximal mappings (Theorem 1 and the dual scheme)."""
import itertools

import numpy as np
import pytest
import scipy.optimize

from oracle import nystrom as ny
from oracle import operators as ops
from oracle import prox as px
from oracle.philox import gaussian_matrix
from workloads import random_kernel


def _small_precond(n, ell, seed, mu=0.0, sqrt_shift=True):
    h = random_kernel(3, seed=seed)
    phi = lambda V: ops.blur_adjoint(ops.blur_apply(V.reshape(-1, n, n), h), h).reshape(V.shape[0], -1)
    r = ny.nystrom(phi, gaussian_matrix(n * n, ell, seed=seed), 2.0 ** -52)
    return ny.Precond(r["U"], r["S_hat"], mu=mu, sqrt_shift=sqrt_shift)


def brute_force_weighted_l1(s, P, tau):
    """argmin_u tau ||u||_1 + 1/2 (u-s)^T P (u-s) by enumerating sign patterns."""
    N = s.size
    Ps = P @ s
    best, best_val = None, np.inf
    for sig in itertools.product((-1, 0, 1), repeat=N):
        sig = np.array(sig, dtype=float)
        S = np.nonzero(sig)[0]
        u = np.zeros(N)
        if S.size:
            u[S] = np.linalg.solve(P[np.ix_(S, S)], Ps[S] - tau * sig[S])
            if np.any(np.sign(u[S]) != sig[S]):
                continue
        val = tau * np.abs(u).sum() + 0.5 * (u - s) @ P @ (u - s)
        if val < best_val:
            best, best_val = u, val
    return best


def test_prox_wavelet_reduces_to_soft_threshold():
    s = np.linspace(-2, 2, 17)
    x, g, it, ok = px.prox_wavelet(s, None, 0.5)
    assert np.allclose(x, np.where(np.abs(s) > 0.5, s - 0.5 * np.sign(s), 0.0))
    x2, _, _, ok2 = px.prox_wavelet(s, np.zeros((2, 17)), 0.5)
    assert ok2 and np.allclose(x2, x)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_prox_wavelet_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    N, r = 6, 2
    Ub = rng.standard_normal((r, N)) * 0.8
    P = np.eye(N) + Ub.T @ Ub
    s = rng.standard_normal(N)
    tau = 0.3
    x, g, it, ok = px.prox_wavelet(s, Ub, tau)
    assert ok
    assert np.allclose(x, brute_force_weighted_l1(s, P, tau), atol=1e-12)


def _bvls_prox(s, Lmat, lam_bar, Pd):
    """Exact prox^P_{lam_bar ||L.||_1}(s) via bounded least squares on the dual."""
    w, V = np.linalg.eigh(Pd)
    Ph = V @ np.diag(np.sqrt(w)) @ V.T
    Pmh = V @ np.diag(1.0 / np.sqrt(w)) @ V.T
    A = lam_bar * Pmh @ Lmat.T
    b = Ph @ s
    res = scipy.optimize.lsq_linear(A, b, bounds=(-1.0, 1.0), method="bvls", tol=1e-14)
    return s - lam_bar * np.linalg.solve(Pd, Lmat.T @ res.x)


def _dense(fn, shape):
    n = int(np.prod(shape))
    return fn(np.eye(n).reshape((n,) + shape)).reshape(n, -1).T


@pytest.mark.parametrize("precond", [False, True])
def test_prox_tv_matches_bvls(precond):
    n = 4
    rng = np.random.default_rng(3)
    s = rng.uniform(size=(n, n))
    lam_bar = 0.15
    P = _small_precond(n, 5, seed=4) if precond else ny.Identity()
    Pd = P.apply(np.eye(n * n)) if precond else np.eye(n * n)
    x_ref = _bvls_prox(s.ravel(), _dense(ops.grad, (n, n)), lam_bar, Pd)
    x, Q = px.prox_dual(s, "tv", lam_bar, P, n_inner=20000)
    assert np.allclose(x.ravel(), x_ref, atol=1e-7)
    assert np.all(np.abs(Q) <= 1.0)


def test_prox_hs_reduces_to_1d_second_difference_tv():
    # s constant along columns -> the HS_1 prox is the 1-D prox of ||D2 f||_1
    n1, n2 = 8, 4
    f = np.random.default_rng(5).uniform(size=n1)
    s = np.tile(f[:, None], (1, n2))
    lam_bar = 0.05
    D2 = _dense(lambda x: np.roll(x, 1, -1) - 2 * x + np.roll(x, -1, -1), (n1,))
    f_ref = _bvls_prox(f, D2, lam_bar, np.eye(n1))
    x, Q = px.prox_dual(s, "hs", lam_bar, ny.Identity(), n_inner=20000)
    assert np.allclose(x, np.tile(f_ref[:, None], (1, n2)), atol=1e-7)


def _hs_primal_dual(s, x, Q, lam_bar, P):
    Pd = P.apply(np.eye(s.size))
    d = (x - s).ravel()
    primal = 0.5 * d @ Pd @ d + lam_bar * px.reg_value(x, "hs")
    LtQ = ops.hess_adjoint(Q).ravel()
    dual = lam_bar * LtQ @ s.ravel() - 0.5 * lam_bar ** 2 * LtQ @ P.inverse(LtQ)
    return primal, dual


def test_prox_hs_duality_gap_closes_with_preconditioner():
    n = 6
    s = np.random.default_rng(7).uniform(size=(n, n))
    P = _small_precond(n, 6, seed=9)
    lam_bar = 0.02
    x, Q = px.prox_dual(s, "hs", lam_bar, P, n_inner=4000)
    primal, dual = _hs_primal_dual(s, x, Q, lam_bar, P)
    assert dual <= primal + 1e-12
    assert primal - dual < 1e-9 * max(1.0, abs(primal))
    # spectral norm of every dual block <= 1
    a, b, c = Q
    r = np.sqrt((0.5 * (a - c)) ** 2 + b * b)
    assert np.all(np.abs(0.5 * (a + c)) + r <= 1.0 + 1e-12)


def test_spectral_projection_matches_eigh():
    rng = np.random.default_rng(11)
    q = rng.standard_normal((3, 5, 7)) * 1.5
    p = px.proj_spectral_2x2(q)
    for i in range(5):
        for j in range(7):
            M = np.array([[q[0, i, j], q[1, i, j]], [q[1, i, j], q[2, i, j]]])
            w, V = np.linalg.eigh(M)
            Mp = V @ np.diag(np.clip(w, -1, 1)) @ V.T
            assert np.allclose([Mp[0, 0], Mp[0, 1], Mp[1, 1]], p[:, i, j], atol=1e-13)
    # a multiple of the identity (r = 0) is clipped on the diagonal only
    z = np.zeros((3, 1, 1))
    z[0] = z[2] = 3.0
    assert np.allclose(px.proj_spectral_2x2(z)[:, 0, 0], [1.0, 0.0, 1.0])
