"""Pins for the oracle's Algorithm 1 and the preconditioner (Eq. RYPreconditioner)."""
import math

import numpy as np
import pytest

from oracle import nystrom as ny
from oracle import operators as ops
from oracle.philox import gaussian_matrix
from workloads import gaussian_kernel, random_kernel

EPS64 = 2.0 ** -52


def dense_phi(phi, n1, n2):
    N = n1 * n2
    eye = np.eye(N).reshape(N, n1, n2)
    return phi(eye).reshape(N, N).T


def flat_phi(phi, n1, n2):
    return lambda V: phi(V.reshape(-1, n1, n2)).reshape(V.shape[0], -1)


def test_exact_recovery_low_rank_operator():
    # blur + 4x decimation on 16x16 has rank <= 16 < ell = 20
    n, d, ell = 16, 4, 20
    h = gaussian_kernel(7, 2.0)
    phi = lambda x: ops.decim_adjoint(ops.decim_apply(x, h, d), h, d)
    Phi = dense_phi(phi, n, n)
    assert np.linalg.matrix_rank(Phi) <= 16
    r = ny.nystrom(flat_phi(phi, n, n), gaussian_matrix(n * n, ell, seed=1), EPS64)
    approx = r["U"].T @ np.diag(r["S_hat"]) @ r["U"]
    assert np.linalg.norm(approx - Phi) <= 1e-9 * np.linalg.norm(Phi)
    assert np.count_nonzero(r["S_hat"] > 1e-9 * r["S_hat"][0]) <= 16


def test_full_sketch_gives_dense_spectrum_and_dft():
    n = 6
    N = n * n
    h = random_kernel(3, seed=2)
    phi = lambda x: ops.blur_adjoint(ops.blur_apply(x, h), h)
    Phi = dense_phi(phi, n, n)
    r = ny.nystrom(flat_phi(phi, n, n), gaussian_matrix(N, N, seed=4), EPS64)
    ev = np.sort(np.linalg.eigvalsh(0.5 * (Phi + Phi.T)))[::-1]
    assert np.allclose(r["S_hat"], np.maximum(ev, 0.0), atol=1e-10)
    pad = np.zeros((n, n))
    for a in range(3):
        for b in range(3):
            pad[(a - 1) % n, (b - 1) % n] = h[a, b]
    sym = np.sort(np.abs(np.fft.fft2(pad)).ravel() ** 2)[::-1]
    assert np.allclose(r["S_hat"], sym, atol=1e-10)


def test_partial_sketch_invariants():
    n, ell = 10, 12
    h = random_kernel(5, seed=3)
    phi = lambda x: ops.blur_adjoint(ops.blur_apply(x, h), h)
    Phi = dense_phi(phi, n, n)
    Om = gaussian_matrix(n * n, ell, seed=8)
    r = ny.nystrom(flat_phi(phi, n, n), Om, EPS64)
    U, S_hat, v = r["U"], r["S_hat"], r["v"]
    assert np.isclose(v, EPS64 * np.linalg.norm(Om))
    # orthonormal columns, descending, nonnegative
    assert np.allclose(U @ U.T, np.eye(ell), atol=1e-12)
    assert np.all(np.diff(S_hat) <= 1e-14) and np.all(S_hat >= 0)
    # Loewner bound: Phi<Omega> <= Phi, so s_i <= lambda_i(Phi)
    ev = np.sort(np.linalg.eigvalsh(Phi))[::-1][:ell]
    assert np.all(S_hat <= ev + 1e-10)
    # B B^T = Y_v (Omega^T Y_v)^{-1} Y_v^T, checked by a plain solve
    Yv = r["Y"] + v * Om
    Mc = Om @ Yv.T
    BBt = Yv.T @ np.linalg.solve(0.5 * (Mc + Mc.T), Yv)
    S2 = S_hat + v                        # S^2 before the shift is removed
    assert np.allclose(U.T @ np.diag(S2) @ U, BBt, atol=1e-10 * np.abs(BBt).max())
    # Nystrom definition (Eq. NYApprox) with the pseudo-inverse, no shift
    Y = r["Y"]
    nys = Y.T @ np.linalg.pinv(Om @ Y.T) @ Y
    assert np.allclose(U.T @ np.diag(S_hat) @ U, nys, atol=1e-8 * np.abs(nys).max())


def test_cholesky_retry_and_failure():
    N, ell = 30, 5
    Om = gaussian_matrix(N, ell, seed=1)
    with pytest.raises(ny.NotSPD):
        ny.nystrom(lambda V: -V, Om, EPS64)
    r = ny.nystrom(lambda V: 0.0 * V, Om, EPS64)          # Phi = 0 is SPSD
    assert r["retries"] == 0 and np.all(r["S_hat"] <= 1e-12)


# ------------------------------------------------------- preconditioner ---

def _factor(seed=0, n=8, ell=10, k=3):
    h = random_kernel(k, seed=seed + 11)
    phi = lambda x: ops.blur_adjoint(ops.blur_apply(x, h), h)
    r = ny.nystrom(flat_phi(phi, n, n), gaussian_matrix(n * n, ell, seed=seed), EPS64)
    return r, dense_phi(phi, n, n)


@pytest.mark.parametrize("sqrt_shift", [False, True])
@pytest.mark.parametrize("mu", [0.0, 1e-2])
def test_precond_inverse_and_min_eigenvalue(sqrt_shift, mu):
    r, _ = _factor()
    P = ny.Precond(r["U"], r["S_hat"], mu=mu, sqrt_shift=sqrt_shift)
    N = r["U"].shape[1]
    Pd = P.apply(np.eye(N))
    Pinv = P.inverse(np.eye(N))
    assert np.allclose(Pd @ Pinv, np.eye(N), atol=1e-12)
    assert np.isclose(np.linalg.eigvalsh(Pd).min(), 1.0)
    assert np.allclose(Pd, np.eye(N) + P.Ubar.T @ P.Ubar, atol=1e-12)


def test_precond_matches_eq_rypreconditioner_unclamped():
    r, _ = _factor(seed=2)
    U, S = r["U"], r["S_hat"]
    mu = 0.05
    sK = S[-1]
    N = U.shape[1]
    P_eq = U.T @ np.diag(S + mu) @ U / (sK + mu) + (np.eye(N) - U.T @ U)
    Pinv_eq = (sK + mu) * U.T @ np.diag(1.0 / (S + mu)) @ U + (np.eye(N) - U.T @ U)
    P = ny.Precond(U, S, mu=mu, sqrt_shift=False)
    assert np.allclose(P.apply(np.eye(N)), P_eq, atol=1e-12)
    assert np.allclose(P.inverse(np.eye(N)), Pinv_eq, atol=1e-12)
    # the last column of Ubar is zero (Sec. III-B)
    assert np.allclose(P.Ubar[-1], 0.0)


def test_precond_identity_when_U_zero_and_degenerate():
    U = np.zeros((3, 20))
    P = ny.Precond(U, np.array([3.0, 2.0, 1.0]))
    z = np.arange(20.0)
    assert np.allclose(P.apply(z), z) and np.allclose(P.inverse(z), z)
    with pytest.raises(ny.Degenerate):
        ny.precond_weights(np.array([1.0, 0.0]), mu=0.0)


def test_theorem2_condition_number_bound():
    # Thm 2: with K = 2 ceil(1.5 d_eff(mu) + 1), E[kappa(P^-1/2 (Phi + mu I) P^-1/2)] < 28
    n = 12
    N = n * n
    h = gaussian_kernel(5, 1.2)
    phi = lambda x: ops.blur_adjoint(ops.blur_apply(x, h), h)
    Phi = dense_phi(phi, n, n)
    mu = 1e-2
    lam = np.linalg.eigvalsh(Phi)
    d_eff = float(np.sum(lam / (lam + mu)))
    K = 2 * math.ceil(1.5 * d_eff + 1)
    assert K < N
    kappas = []
    for seed in range(20):
        r = ny.nystrom(flat_phi(phi, n, n), gaussian_matrix(N, K, seed=100 + seed), EPS64)
        P = ny.Precond(r["U"], r["S_hat"], mu=mu, sqrt_shift=False)
        Pinv = P.inverse(np.eye(N))
        w, V = np.linalg.eigh(0.5 * (Pinv + Pinv.T))
        Pmh = V @ np.diag(np.sqrt(w)) @ V.T
        ev = np.linalg.eigvalsh(Pmh @ (Phi + mu * np.eye(N)) @ Pmh)
        kappas.append(ev.max() / ev.min())
    assert np.mean(kappas) < 28.0
    # and the preconditioner helps
    assert np.mean(kappas) < (lam.max() + mu) / (lam.min() + mu)
