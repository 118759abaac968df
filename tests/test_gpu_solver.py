"""GPU parity of Algorithm 3 (WAPG / APG) against the float64 oracle after a fixed
number of iterations, with the same U, S_hat and step size fed to both."""
import math

import numpy as np
import pytest

import oracle
from oracle import operators as O
from oracle.philox import gaussian_matrix
from workloads import gaussian_kernel, phantom
from tests.gpu_util import rel, require_gpu

pytestmark = pytest.mark.gpu
EPS64 = 2.0 ** -52


@pytest.fixture(scope="module")
def env():
    torch, api = require_gpu()
    return torch, api, api.Context(0)


def _setup(kind, n, ell, seed, reg, lam, fit="l2", delta=0.0, decim=1, na=0, nb=0, ksize=9, sigma=1.5,
           levels=3, noise=0.01, wavelet="haar"):
    h = gaussian_kernel(ksize, sigma) if kind != "radon" else None
    opo = O.Operator(kind, n, n, kernel=h, decim=decim, n_angles=na, n_bins=nb)
    x_true = phantom(n, 8, seed, "mixed")
    y = opo.apply(x_true)
    y = y + np.random.default_rng(seed + 1).normal(0, noise * max(1.0, np.abs(y).max()), y.shape)
    prob = oracle.wapg.Problem(opo, y, lam, reg, fit=fit, huber_delta=delta, haar_levels=levels, wavelet=wavelet)
    phi = lambda V: prob.phi(V.reshape(-1, n, n)).reshape(V.shape[0], -1)
    ref = oracle.nystrom.nystrom(phi, gaussian_matrix(n * n, ell, seed + 2), EPS64) if ell else None
    return h, opo, prob, y, ref


def _run(env, dt, kind, n, ell, reg, lam, iters, n_inner=10, fit="l2", delta=0.0, decim=1, na=0, nb=0,
         levels=3, seed=1, precond=True, wavelet="haar"):
    torch, api, ctx = env
    h, opo, prob, y, ref = _setup(kind, n, ell if precond else 0, seed, reg, lam, fit, delta, decim, na, nb,
                                  levels=levels, wavelet=wavelet)
    P = oracle.nystrom.Precond(ref["U"], ref["S_hat"]) if precond else None
    alpha = 1.0 / oracle.wapg.power_lipschitz(prob, P)
    x_ref = prob.to_image(oracle.wapg.wapg(prob, alpha, iters, precond=P, n_inner=n_inner)["x"])
    tdt = torch.float64 if dt == "f64" else torch.float32
    op = api.Operator(ctx, kind, n, n, dtype=tdt, kernel=h, decim=decim, n_angles=na, n_bins=nb,
                      haar_levels=levels if reg == "wavelet" else 0, wavelet=wavelet)
    pc = None
    if precond:
        pc = api.Precond(ctx, n * n, ell, tdt).import_factor(ref["U"], ref["S_hat"], 0.0, True)
    sol = api.Solver(ctx, op, torch.from_numpy(y).to(tdt).cuda(), reg, lam, pc=pc, fit=fit, huber_delta=delta,
                     alpha=alpha, n_inner=n_inner)
    sol.step(iters)
    return rel(sol.x().cpu(), x_ref)


def test_wapg_wavelet_deblur64_f64(env):
    # the 64 x 64 float64 deblurring workload: 9 x 9 sigma 1.5, Haar-3, lambda 1e-3, ell 32
    assert _run(env, "f64", "blur", 64, 32, "wavelet", 1e-3, 15) < 1e-9


@pytest.mark.parametrize("dt,tol", [("f64", 1e-9)])
def test_wapg_daubechies4_deblur(env, dt, tol):
    # the wavelet model with the four-tap Daubechies transform (4 levels, the
    # CT experiments' choice): Phi = W A^T A W^T sketched by the oracle, the
    # semi-smooth Newton prox, 15 WAPG iterations
    assert _run(env, dt, "blur", 64, 32, "wavelet", 1e-3, 15, levels=4, wavelet="db4") < tol


def test_apg_plain_tv_f64(env):
    assert _run(env, "f64", "blur", 48, 0, "tv", 5e-3, 12, precond=False) < 1e-10


@pytest.mark.parametrize("dt,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_wapg_tv_blur(env, dt, tol):
    assert _run(env, dt, "blur", 64, 16, "tv", 5e-3, 20) < tol


def test_wapg_hs_huber_superres_f32(env):
    assert _run(env, "f32", "blur_decim", 64, 12, "hs", 1e-3, 15, fit="huber", delta=0.01, decim=4) < 1e-4


@pytest.mark.parametrize("reg,dt,tol", [("isotv", "f64", 1e-10), ("isotv", "f32", 1e-4), ("hs2", "f64", 1e-10),
                                         ("hsinf", "f64", 1e-10)])
def test_wapg_mixed_norm_variants_blur(env, reg, dt, tol):
    assert _run(env, dt, "blur", 64, 16, reg, 5e-3, 15) < tol


def test_wapg_tv_fanbeam_f64(env):
    # Algorithm 3 on the fan-beam forward model (Sketch, factor and the
    # P-metric TV prox unchanged): 10 iterations against the oracle
    torch, api, ctx = env
    n, A, B, R, D, ell, lam = 32, 24, 64, 40.0, 80.0, 16, 2e-3
    opo = O.Operator("fanbeam", n, n, n_angles=A, n_bins=B, src_dist=R, det_dist=D, det_spacing=1.0)
    x_true = phantom(n, 6, 4, "mixed")
    y = opo.apply(x_true)
    y = y + np.random.default_rng(5).normal(0, 0.01 * np.abs(y).max(), y.shape)
    prob = oracle.wapg.Problem(opo, y, lam, "tv")
    phi = lambda V: prob.phi(V.reshape(-1, n, n)).reshape(V.shape[0], -1)
    ref = oracle.nystrom.nystrom(phi, gaussian_matrix(n * n, ell, 6), EPS64)
    P = oracle.nystrom.Precond(ref["U"], ref["S_hat"])
    alpha = 1.0 / oracle.wapg.power_lipschitz(prob, P)
    x_ref = oracle.wapg.wapg(prob, alpha, 10, precond=P, n_inner=10)["x"]
    op = api.Operator(ctx, "fanbeam", n, n, dtype=torch.float64, n_angles=A, n_bins=B, src_dist=R, det_dist=D)
    pc = api.Precond(ctx, n * n, ell, torch.float64).import_factor(ref["U"], ref["S_hat"], 0.0, True)
    sol = api.Solver(ctx, op, torch.from_numpy(y).cuda(), "tv", lam, pc=pc, alpha=alpha, n_inner=10)
    sol.step(10)
    assert rel(sol.x().cpu(), x_ref) < 1e-10


def test_wapg_tv_radon_f32(env):
    assert _run(env, "f32", "radon", 48, 16, "tv", 2e-4, 10, na=30, nb=70) < 1e-4


def test_step_size_estimate_close_to_oracle(env):
    torch, api, ctx = env
    h, opo, prob, y, ref = _setup("blur", 64, 16, 3, "tv", 5e-3)
    P = oracle.nystrom.Precond(ref["U"], ref["S_hat"])
    a_ref = 1.0 / oracle.wapg.power_lipschitz(prob, P)
    op = api.Operator(ctx, "blur", 64, 64, dtype=torch.float64, kernel=h)
    pc = api.Precond(ctx, 64 * 64, 16, torch.float64).import_factor(ref["U"], ref["S_hat"], 0.0, True)
    sol = api.Solver(ctx, op, torch.from_numpy(y).cuda(), "tv", 5e-3, pc=pc)
    assert abs(sol.alpha - a_ref) <= 0.02 * a_ref


@pytest.mark.parametrize("reg,fit,dt", [("tv", "l2", "f64"), ("hs", "huber", "f64"), ("wavelet", "l2", "f64"),
                                        ("tv", "l2", "f32"), ("isotv", "l2", "f64"), ("hs2", "l2", "f64"),
                                        ("hsinf", "huber", "f64")])
def test_objective_matches_oracle(env, reg, fit, dt):
    torch, api, ctx = env
    n = 48
    h, opo, prob, y, ref = _setup("blur", n, 0, 6, reg, 3e-3, fit=fit, delta=0.02, levels=2)
    tdt = torch.float64 if dt == "f64" else torch.float32
    op = api.Operator(ctx, "blur", n, n, dtype=tdt, kernel=h, haar_levels=2 if reg == "wavelet" else 0)
    alpha = 1.0 / oracle.wapg.power_lipschitz(prob)
    sol = api.Solver(ctx, op, torch.from_numpy(y).to(tdt).cuda(), reg, 3e-3, fit=fit, huber_delta=0.02,
                     alpha=alpha, n_inner=10)
    sol.step(7)
    xv = oracle.wapg.wapg(prob, alpha, 7, n_inner=10)["x"]
    F_ref = prob.objective(xv)
    assert abs(sol.objective() - F_ref) <= (1e-10 if dt == "f64" else 1e-5) * abs(F_ref)


@pytest.mark.parametrize("reg,dt", [("tv", "f32"), ("hs", "f64"), ("wavelet", "f64")])
def test_graph_replay_matches_direct_launches(env, reg, dt):
    # the captured even/odd iteration graphs give the same iterates as
    # launching every kernel one by one, across odd step counts and restarts
    torch, api, ctx = env
    n = 64
    h, opo, prob, y, ref = _setup("blur", n, 16, 2, reg, 2e-3, levels=3)
    tdt = torch.float64 if dt == "f64" else torch.float32
    op = api.Operator(ctx, "blur", n, n, dtype=tdt, kernel=h, haar_levels=3 if reg == "wavelet" else 0)
    pc = api.Precond(ctx, n * n, 16, tdt).import_factor(ref["U"], ref["S_hat"], 0.0, True)
    yt = torch.from_numpy(y).to(tdt).cuda()
    a = api.Solver(ctx, op, yt, reg, 2e-3, pc=pc, n_inner=8, use_graph=True)
    b = api.Solver(ctx, op, yt, reg, 2e-3, pc=pc, n_inner=8, use_graph=False)
    for steps in (3, 4, 1):
        a.step(steps)
        b.step(steps)
    assert rel(a.x().cpu(), b.x().cpu()) == 0.0
    a.restart(True)
    b.restart(True)
    a.step(5)
    b.step(5)
    assert rel(a.x().cpu(), b.x().cpu()) == 0.0


def test_end_to_end_gpu_sketch_reaches_same_minimiser(env):
    # sketch + factor on the device; preconditioned and plain runs approach the
    # same minimiser (Sec. III-B: P changes the metric, not the solution)
    torch, api, ctx = env
    n = 48
    h = gaussian_kernel(9, 1.5)
    opo = O.Operator("blur", n, n, kernel=h)
    y = opo.apply(phantom(n, 8, 4, "mixed")) + np.random.default_rng(5).normal(0, 0.01, (n, n))
    op = api.Operator(ctx, "blur", n, n, dtype=torch.float64, kernel=h)
    Om, Y = api.nys_sketch(ctx, op, 24, seed=9)
    pc = api.nys_factor(ctx, Om, Y, EPS64)
    yt = torch.from_numpy(y).cuda()
    a = api.Solver(ctx, op, yt, "tv", 5e-3, pc=pc, n_inner=20)
    b = api.Solver(ctx, op, yt, "tv", 5e-3, pc=None, n_inner=20)
    a.step(3000)
    b.step(3000)
    assert rel(a.x().cpu(), b.x().cpu()) < 1e-4


def test_solver_graph_recaptured_after_workspace_growth(env):
    # A float32 solver replays the CUDA graph of its iteration.  A float64
    # solver created afterwards on the same context needs larger scratch
    # regions (its dual variables and partial sums take twice the bytes), so
    # the context reallocates them and frees the old ones.  The first solver
    # must capture its graph again rather than replay the freed addresses: its
    # iterates equal those of the same solver run alone on a fresh context.
    torch, api, ctx = env
    n, ell, lam = 64, 16, 5e-3
    h, opo, prob, y, ref = _setup("blur", n, ell, 3, "tv", lam)
    P = oracle.nystrom.Precond(ref["U"], ref["S_hat"])
    alpha = 1.0 / oracle.wapg.power_lipschitz(prob, P)

    def solver(c, dtype):
        op = api.Operator(c, "blur", n, n, dtype=dtype, kernel=h)
        pc = api.Precond(c, n * n, ell, dtype).import_factor(ref["U"], ref["S_hat"], 0.0, True)
        return op, pc, api.Solver(c, op, torch.from_numpy(y).to(dtype).cuda(), "tv", lam, pc=pc, alpha=alpha,
                                  n_inner=10)

    fresh = api.Context(0)
    ctx_a = api.Context(0)
    keep_a = solver(ctx_a, torch.float32)
    keep_a[2].step(4)
    keep_b = solver(ctx_a, torch.float64)      # grows the shared workspace
    keep_b[2].step(2)
    keep_a[2].step(4)
    keep_c = solver(fresh, torch.float32)
    keep_c[2].step(8)
    assert rel(keep_a[2].x().cpu(), keep_c[2].x().cpu()) < 1e-6
