"""Pins for the oracle's Algorithm 3 (WAPG / APG) against optimality and rate theory."""
import numpy as np
import pytest

from oracle import nystrom as ny
from oracle import operators as ops
from oracle import wapg as wp
from oracle.philox import gaussian_matrix
from workloads import gaussian_kernel, phantom


def _wavelet_problem(n=16, lam=1e-2, seed=1):
    h = gaussian_kernel(5, 1.0)
    op = ops.Operator("blur", n, n, kernel=h)
    x_true = phantom(n, 4, seed, "mixed")
    y = op.apply(x_true) + np.random.default_rng(seed + 1).normal(0, 0.01, (n, n))
    return wp.Problem(op, y, lam, "wavelet", haar_levels=2)


def _precond_for(prob, ell, seed=3, sqrt_shift=True, mu=0.0):
    n1, n2 = prob.shape
    phi = lambda V: prob.phi(V.reshape(-1, n1, n2)).reshape(V.shape[0], -1)
    r = ny.nystrom(phi, gaussian_matrix(n1 * n2, ell, seed=seed), 2.0 ** -52)
    return ny.Precond(r["U"], r["S_hat"], mu=mu, sqrt_shift=sqrt_shift), r


def _lasso_certificate(prob, xbar):
    """Optimality of min 1/2||A W^T xbar - y||^2 + lam ||xbar||_1: 0 in grad + lam d|.|."""
    g = prob.grad_f(xbar).ravel()
    xb = xbar.ravel()
    on = np.abs(xb) > 1e-10
    viol_on = np.abs(g[on] + prob.lam * np.sign(xb[on]))
    viol_off = np.maximum(np.abs(g[~on]) - prob.lam, 0.0)
    return max(viol_on.max(initial=0.0), viol_off.max(initial=0.0))


def test_wavelet_same_minimiser_with_and_without_preconditioner():
    prob = _wavelet_problem()
    P, _ = _precond_for(prob, 24)
    a_plain = 1.0 / wp.power_lipschitz(prob)
    a_prec = 1.0 / wp.power_lipschitz(prob, P)
    x_plain = wp.wapg(prob, a_plain, 3000)["x"]
    x_prec = wp.wapg(prob, a_prec, 3000, precond=P)["x"]
    assert _lasso_certificate(prob, x_plain) < 1e-6
    assert _lasso_certificate(prob, x_prec) < 1e-6
    assert np.linalg.norm(x_plain - x_prec) <= 1e-6 * np.linalg.norm(x_plain)


def test_wapg_rate_bound_and_monotone_pgd():
    prob = _wavelet_problem(lam=2e-2, seed=5)
    P, _ = _precond_for(prob, 24, seed=6)
    Lhat = wp.power_lipschitz(prob, P)
    x_star = wp.wapg(prob, 1.0 / Lhat, 4000, precond=P)["x"]
    F_star = prob.objective(x_star)
    d = x_star.ravel()                     # x^1 = 0
    bound_num = 2.0 * Lhat * d @ P.apply(d)
    F = []
    wp.wapg(prob, 1.0 / Lhat, 60, precond=P, callback=lambda k, x: F.append(prob.objective(x)))
    for k, Fk in enumerate(F, start=1):
        assert Fk - F_star <= bound_num / (k + 1) ** 2 + 1e-12
    # without momentum the P-metric proximal gradient decreases F monotonically
    G = []
    wp.wapg(prob, 1.0 / Lhat, 60, precond=P, momentum=False,
            callback=lambda k, x: G.append(prob.objective(x)))
    assert np.all(np.diff(G) <= 1e-12 * abs(G[0]))


def test_full_rank_sketch_solves_least_squares_in_one_step():
    # lambda = 0, ell = N, no square-root heuristic: P^{-1} Phi = s_N I on R^N
    n = 6
    h = gaussian_kernel(3, 0.7)
    op = ops.Operator("blur", n, n, kernel=h)
    y = np.random.default_rng(2).standard_normal((n, n))
    prob = wp.Problem(op, y, 0.0, "wavelet", haar_levels=1)
    P, r = _precond_for(prob, n * n, seed=4, sqrt_shift=False)
    alpha = 1.0 / r["S_hat"][-1]
    x1 = wp.wapg(prob, alpha, 1, precond=P)["x"]
    Phi = np.array([prob.phi(e.reshape(n, n)).ravel() for e in np.eye(n * n)]).T
    b = -prob.grad_f(np.zeros((n, n))).ravel()
    x_star = np.linalg.solve(Phi, b)
    assert np.allclose(x1.ravel(), x_star, atol=1e-8 * np.abs(x_star).max())


@pytest.mark.parametrize("reg", ["tv", "hs"])
def test_dual_prox_wapg_same_minimiser(reg):
    n = 10
    h = gaussian_kernel(3, 0.8)
    op = ops.Operator("blur", n, n, kernel=h)
    x_true = phantom(n, 3, 4, "mixed")
    y = op.apply(x_true) + np.random.default_rng(9).normal(0, 0.01, (n, n))
    prob = wp.Problem(op, y, 5e-3, reg)
    P, _ = _precond_for(prob, 12, seed=8)
    x_plain = wp.wapg(prob, 1.0 / wp.power_lipschitz(prob), 1500, n_inner=20)["x"]
    x_prec = wp.wapg(prob, 1.0 / wp.power_lipschitz(prob, P), 1500, precond=P, n_inner=20)["x"]
    assert np.linalg.norm(x_plain - x_prec) <= 1e-5 * np.linalg.norm(x_plain)
    # both lower the objective below that of the data itself
    assert prob.objective(x_prec) < prob.objective(y)


def _huber_problem(delta, n=10, seed=4):
    rng = np.random.default_rng(seed)
    op = ops.Operator("blur_decim", n, n, kernel=gaussian_kernel(3, 1.0), decim=2)
    y = op.apply(phantom(n, 3, seed, "mixed")) + rng.normal(0, 0.05, (n // 2, n // 2))
    return wp.Problem(op, y, 0.0, "tv", fit="huber", huber_delta=delta), rng


def test_huber_gradient_is_the_derivative_of_its_objective():
    # lambda = 0 isolates the data term; central differences along random
    # directions, with the residuals spread across both sides of delta
    prob, rng = _huber_problem(0.03)
    x = rng.uniform(0, 1, prob.shape)
    r = np.abs(prob.op.apply(x) - prob.y)
    assert (r <= 0.03).any() and (r > 0.03).any()
    g = prob.grad_f(x)
    for _ in range(5):
        d = rng.standard_normal(prob.shape)
        h = 1e-6
        fd = (prob.objective(x + h * d) - prob.objective(x - h * d)) / (2 * h)
        assert np.sum(g * d) == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_huber_limits():
    # delta above every residual: least squares; delta -> 0: h/delta -> |r|
    prob, rng = _huber_problem(1e6)
    x = rng.uniform(0, 1, prob.shape)
    ls = wp.Problem(prob.op, prob.y, 0.0, "tv")
    assert prob.objective(x) == pytest.approx(ls.objective(x), rel=1e-14)
    assert np.allclose(prob.grad_f(x), ls.grad_f(x), rtol=1e-14, atol=0)
    small, _ = _huber_problem(1e-9)
    r = small.op.apply(x) - small.y
    assert small.objective(x) / 1e-9 == pytest.approx(np.abs(r).sum(), rel=1e-6)


def test_huber_objective_is_the_integral_of_its_gradient():
    # F(x1) - F(x0) = int_0^1 <grad F(x0 + t (x1 - x0)), x1 - x0> dt along a
    # path whose residuals cross delta: a jump between the quadratic and the
    # linear branch (a wrong constant) breaks it
    prob, rng = _huber_problem(0.03)
    x0, x1 = rng.uniform(0, 1, prob.shape), rng.uniform(0, 1, prob.shape)
    d = x1 - x0
    t = np.linspace(0.0, 1.0, 4001)
    vals = np.array([np.sum(prob.grad_f(x0 + s * d) * d) for s in t])
    integral = np.sum(0.5 * (vals[1:] + vals[:-1]) * np.diff(t))
    r0 = np.abs(prob.op.apply(x0) - prob.y)
    r1 = np.abs(prob.op.apply(x1) - prob.y)
    assert ((r0 <= 0.03) != (r1 <= 0.03)).any()
    assert prob.objective(x1) - prob.objective(x0) == pytest.approx(integral, rel=1e-6)


@pytest.mark.parametrize("sqrt_shift", [None, False, True])
def test_power_lipschitz_is_the_largest_eigenvalue_of_pinv_phi(sqrt_shift):
    # Algorithm 3's step size needs L_f^P = lambda_max(P^{-1} Phi).  Its
    # eigenvalues are those of the pencil Phi v = lambda P v, solved here by a
    # dense generalised symmetric eigensolver with P assembled column by column
    # from P.apply (no use of P.inverse): the estimate must be 1.02 times the
    # top one.  An estimate of P Phi (apply and inverse swapped) is 8-50 times
    # off on this problem, and a missing safety factor 2 % off.
    import scipy.linalg
    n = 8
    op = ops.Operator("blur", n, n, kernel=gaussian_kernel(5, 1.0))
    prob = wp.Problem(op, op.apply(phantom(n, 3, 2, "mixed")), 1e-3, "tv")
    dense = lambda f: np.array([f(e.reshape(n, n)).ravel() for e in np.eye(n * n)]).T
    Phi = dense(prob.phi)
    if sqrt_shift is None:
        P, Pd = None, np.eye(n * n)
    else:
        P, _ = _precond_for(prob, 10, seed=5, sqrt_shift=sqrt_shift)
        assert (P.d > 0).sum() >= 5
        Pd = dense(P.apply)
    lam_max = scipy.linalg.eigh(Phi, Pd, eigvals_only=True)[-1]
    assert wp.power_lipschitz(prob, P, iters=1000) == pytest.approx(1.02 * lam_max, rel=1e-12)
    assert wp.power_lipschitz(prob, P) == pytest.approx(1.02 * lam_max, rel=1e-4)
