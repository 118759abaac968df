"""GPU parity of Algorithm 1 (sketch + factor), the preconditioner and the proxes
against the float64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from oracle import operators as O
from oracle.philox import gaussian_matrix
from workloads import gaussian_kernel, gaussian_probe_like, phantom
from tests.gpu_util import TOL, close, rel, require_gpu

pytestmark = pytest.mark.gpu
EPS64 = 2.0 ** -52
EPS32 = 2.0 ** -23


@pytest.fixture(scope="module")
def env():
    torch, api = require_gpu()
    return torch, api, api.Context(0)


def _flat_phi(opo, n1, n2):
    return lambda V: opo.normal(V.reshape(-1, n1, n2)).reshape(V.shape[0], -1)


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("N,ell", [(64 * 64, 32), (37 * 29, 7), (5, 3)])
def test_omega_matches_philox_spec(env, dt, N, ell):
    torch, api, ctx = env
    n1 = {4096: 64, 1073: 37, 5: 1}[N]
    n2 = N // n1
    tdt = torch.float64 if dt == "f64" else torch.float32
    op = api.Operator(ctx, "blur", n1, n2, dtype=tdt, kernel=np.ones((1, 1)))
    Om, Y = api.nys_sketch(ctx, op, ell, seed=0x1234_5678_9ABC)
    ref = gaussian_matrix(N, ell, 0x1234_5678_9ABC)
    got = Om.reshape(ell, N).double().cpu().numpy()
    assert np.max(np.abs(got - ref)) <= (1e-13 if dt == "f64" else 4e-6) * max(1.0, np.abs(ref).max())
    # 1 x 1 unit kernel: Phi = I
    assert np.array_equal(Y.cpu().numpy(), Om.cpu().numpy())


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_sketch_blur_and_wavelet(env, dt):
    torch, api, ctx = env
    n, ell = 64, 12
    h = gaussian_kernel(9, 1.5)
    tdt = torch.float64 if dt == "f64" else torch.float32
    op = api.Operator(ctx, "blur", n, n, dtype=tdt, kernel=h, haar_levels=3)
    opo = O.Operator("blur", n, n, kernel=h)
    Om_ref = gaussian_matrix(n * n, ell, 3).reshape(ell, n, n)
    _, Y = api.nys_sketch(ctx, op, ell, seed=3)
    assert rel(Y.cpu(), opo.normal(Om_ref)) < TOL[dt]
    _, Yw = api.nys_sketch(ctx, op, ell, seed=3, phi="w_ata_wt")
    ref = O.haar_forward(opo.normal(O.haar_adjoint(Om_ref, 3)), 3)
    assert rel(Yw.cpu(), ref) < TOL[dt]


def _check_factor(U_g, S_g, ref, rtol_s, rtol_op):
    # eigenvalues, and the low-rank operator U S U^T on random vectors (basis-free)
    S_ref = ref["S_hat"]
    assert np.max(np.abs(S_g - S_ref)) <= rtol_s * S_ref[0]
    Z = np.random.default_rng(1).standard_normal((5, U_g.shape[1]))
    A_g = ((Z @ U_g.T) * S_g) @ U_g
    A_r = ((Z @ ref["U"].T) * S_ref) @ ref["U"]
    assert rel(A_g, A_r) < rtol_op


def test_factor_f64_matches_algorithm1(env):
    torch, api, ctx = env
    n, ell = 64, 32
    h = gaussian_kernel(9, 1.5)
    op = api.Operator(ctx, "blur", n, n, dtype=torch.float64, kernel=h)
    opo = O.Operator("blur", n, n, kernel=h)
    Om, Y = api.nys_sketch(ctx, op, ell, seed=3)
    pc = api.nys_factor(ctx, Om, Y, EPS64)
    ref = oracle.nystrom.nystrom(_flat_phi(opo, n, n), gaussian_matrix(n * n, ell, 3), EPS64)
    assert abs(pc.v - ref["v"]) <= 1e-12 * ref["v"] and pc.chol_retries == ref["retries"]
    _check_factor(pc.U.cpu().numpy(), pc.S_hat.cpu().numpy(), ref, 1e-10, 1e-9)
    # orthonormal columns
    U = pc.U.cpu().numpy()
    assert np.max(np.abs(U @ U.T - np.eye(ell))) < 1e-9


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("ell", [1, 2, 3])
def test_tiny_sketches_end_to_end(env, dt, ell):
    # the smallest sketches: Algorithm 1 (a 1 x 1 core has one eigenvalue),
    # the preconditioner (the square-root heuristic; the unit-sum blur has
    # S_hat <= 1, so d_ell = sqrt(s_ell) - 1 <= 0 and ell = 1 leaves no
    # active column: P = I exactly) and the P-metric TV prox
    torch, api, ctx = env
    n = 24
    h = gaussian_kernel(5, 1.0)
    idt = torch.float64 if dt == "f64" else torch.float32
    sd = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dt]
    op = api.Operator(ctx, "blur", n, n, dtype=idt, kernel=h)
    opo = O.Operator("blur", n, n, kernel=h)
    eps = EPS64 if dt == "f64" else EPS32
    Om, Y = api.nys_sketch(ctx, op, ell, seed=5, store_dtype=sd)
    pc = api.nys_factor(ctx, Om, Y, eps, u_dtype=sd)
    ref = oracle.nystrom.nystrom(_flat_phi(opo, n, n), gaussian_matrix(n * n, ell, 5), eps)
    tol = {"f64": (1e-10, 1e-9), "f32": (1e-4, 1e-3), "bf16": (3e-2, 3e-2)}[dt]
    _check_factor(pc.U.double().cpu().numpy(), pc.S_hat.cpu().numpy(), ref, *tol)
    d = oracle.nystrom.precond_weights(pc.S_hat.cpu().numpy(), 0.0, True)
    assert pc.ell_active == int(np.sum(d > 0)) and d[-1] == 0.0
    Ul = pc.U.double().cpu().numpy().reshape(ell, -1)
    P = oracle.nystrom.Precond(Ul, pc.S_hat.cpu().numpy(), 0.0, True)
    s = gaussian_probe_like((n, n), 6)
    x_ref, _ = oracle.prox.prox_dual(s, "tv", 0.05, P, 5)
    x, _ = api.prox_tv(ctx, pc, 0.05, 5, torch.from_numpy(s).to(idt).cuda())
    ptol = 1e-10 if dt == "f64" else 1e-4
    close(x, x_ref, ptol, 10 * ptol)


def test_factor_f32_and_bf16_stated_accuracy(env):
    torch, api, ctx = env
    n, ell = 128, 48
    h = gaussian_kernel(9, 1.5)
    op = api.Operator(ctx, "blur", n, n, dtype=torch.float32, kernel=h)
    opo = O.Operator("blur", n, n, kernel=h)
    ref = oracle.nystrom.nystrom(_flat_phi(opo, n, n), gaussian_matrix(n * n, ell, 4), EPS32)
    Om, Y = api.nys_sketch(ctx, op, ell, seed=4)
    pc = api.nys_factor(ctx, Om, Y, EPS32)
    _check_factor(pc.U.double().cpu().numpy(), pc.S_hat.cpu().numpy(), ref, 1e-4, 1e-3)
    Ob, Yb = api.nys_sketch(ctx, op, ell, seed=4, store_dtype=torch.bfloat16)
    pcb = api.nys_factor(ctx, Ob, Yb, EPS32, u_dtype=torch.bfloat16)
    _check_factor(pcb.U.double().cpu().numpy(), pcb.S_hat.cpu().numpy(), ref, 3e-2, 3e-2)


@pytest.mark.parametrize("dt,ell", [("f32", 300), ("f64", 200)])
def test_factor_large_ell_global_jacobi(env, dt, ell):
    # sketch sizes whose ell x ell core does not fit in shared memory (float32
    # above 236, float64 above 166): float64 Cholesky of the core, one-sided
    # Jacobi with R in global memory
    torch, api, ctx = env
    n = 64
    h = gaussian_kernel(9, 1.5)
    tdt = torch.float64 if dt == "f64" else torch.float32
    eps = EPS64 if dt == "f64" else EPS32
    op = api.Operator(ctx, "blur", n, n, dtype=tdt, kernel=h)
    opo = O.Operator("blur", n, n, kernel=h)
    ref = oracle.nystrom.nystrom(_flat_phi(opo, n, n), gaussian_matrix(n * n, ell, 5), eps)
    Om, Y = api.nys_sketch(ctx, op, ell, seed=5)
    pc = api.nys_factor(ctx, Om, Y, eps)
    tol = (1e-9, 1e-8) if dt == "f64" else (1e-4, 1e-3)
    _check_factor(pc.U.double().cpu().numpy(), pc.S_hat.cpu().numpy(), ref, *tol)


@pytest.mark.parametrize("ell", [256, 257, 300, 448, 520])
def test_factor_bf16_wide_sketch_matches_oracle(env, ell):
    # bf16 sketches at and past one 256-column tensor-core tile: the single
    # launch of Omega^T Omega, Omega^T Y, Y^T Y and the tall U = Y_v W in
    # column blocks; the cluster eigensolver on 8 CTAs (256), on 16 (257 ..
    # 448, its upper end) and the global-memory one beyond (520); against the
    # oracle from the same Omega at the bf16 tolerance
    torch, api, ctx = env
    n = 64
    h = gaussian_kernel(9, 1.5)
    op = api.Operator(ctx, "blur", n, n, dtype=torch.float32, kernel=h)
    opo = O.Operator("blur", n, n, kernel=h)
    ref = oracle.nystrom.nystrom(_flat_phi(opo, n, n), gaussian_matrix(n * n, ell, 8), EPS32)
    Ob, Yb = api.nys_sketch(ctx, op, ell, seed=8, store_dtype=torch.bfloat16)
    pcb = api.nys_factor(ctx, Ob, Yb, EPS32, u_dtype=torch.bfloat16)
    _check_factor(pcb.U.double().cpu().numpy(), pcb.S_hat.cpu().numpy(), ref, 3e-2, 3e-2)


@pytest.mark.parametrize("sd,tol", [("f32", 2e-4), ("bf16", 2e-2)])
def test_factor_full_size_properties(env, sd, tol):
    # the 512 x 512, ell = 200, 25 x 25 sigma 4 sketch in the bench's launch
    # configuration.  Properties that hold at any size: B B^T Omega = Y_v, i.e.
    # U (S_hat + v) U^T Omega = Y + v Omega on the sketched columns; U^T U = I;
    # 0 <= s_i <= lambda_max(A^T A) = 1; descending order.
    torch, api, ctx = env
    n, ell = 512, 200
    op = api.Operator(ctx, "blur", n, n, dtype=torch.float32, kernel=gaussian_kernel(25, 4.0))
    tsd = torch.bfloat16 if sd == "bf16" else torch.float32
    Om, Y = api.nys_sketch(ctx, op, ell, seed=13, store_dtype=tsd)
    pc = api.nys_factor(ctx, Om, Y, EPS32, u_dtype=tsd)
    U = pc.U.double()
    S = pc.S_hat
    assert torch.all(S[:-1] >= S[1:]) and S[-1] >= 0 and S[0] <= 1.0 + 1e-3
    G = U @ U.T
    assert torch.max(torch.abs(G - torch.eye(ell, dtype=torch.float64, device=G.device))).item() < 50 * tol
    cols = [0, 7, 99, 199]
    Oc = Om.reshape(ell, -1)[cols].double()
    Yc = Y.reshape(ell, -1)[cols].double()
    lhs = ((Oc @ U.T) * (S + pc.v)) @ U
    rhs = Yc + pc.v * Oc
    assert rel(lhs.cpu(), rhs.cpu()) < tol


def test_exact_recovery_low_rank_on_gpu(env):
    # blur + 4x decimation of a 16 x 16 image has rank <= 16 < ell = 20
    torch, api, ctx = env
    n, d, ell = 16, 4, 20
    h = gaussian_kernel(7, 2.0)
    op = api.Operator(ctx, "blur_decim", n, n, dtype=torch.float64, kernel=h, decim=d)
    Om, Y = api.nys_sketch(ctx, op, ell, seed=5)
    pc = api.nys_factor(ctx, Om, Y, EPS64)
    U, S = pc.U.cpu().numpy(), pc.S_hat.cpu().numpy()
    opo = O.Operator("blur_decim", n, n, kernel=h, decim=d)
    Phi = opo.normal(np.eye(n * n).reshape(-1, n, n)).reshape(n * n, -1)
    assert np.linalg.norm(U.T @ np.diag(S) @ U - Phi) <= 1e-9 * np.linalg.norm(Phi)


def test_not_spd_core_is_reported(env):
    # Y = -Omega is the sketch of Phi = -I: the shifted core stays negative definite
    torch, api, ctx = env
    from paper_2411_08178_gb300._abi import NYS_ENOTSPD, NysError
    Om = torch.from_numpy(gaussian_matrix(400, 6, 1).reshape(6, 20, 20)).cuda()
    with pytest.raises(NysError) as e:
        api.nys_factor(ctx, Om, -Om, EPS64)
    assert e.value.code == NYS_ENOTSPD


@pytest.mark.parametrize("ell", [6, 47, 48, 64, 200, 512, 513])
def test_cholesky_retries_match_oracle(env, ell):
    # Y = -delta Omega: the core (v - delta) Omega^T Omega is SPD only once the
    # shift v = eps ||Omega||_F, multiplied by 10 per failure, exceeds delta.
    # delta = 10^2.5 v0 needs three retries; the count, the final shift and the
    # factor against the oracle's Algorithm 1 with the same retry rule.  ell =
    # 48 .. 512 run the 16-SM cluster Cholesky (both ends of its range), 6, 47
    # and 513 the one-CTA kernel.
    torch, api, ctx = env
    n = 32 if ell <= 512 else 24
    Om = torch.from_numpy(gaussian_matrix(n * n, ell, 11).reshape(ell, n, n)).cuda()
    v0 = EPS64 * float(torch.linalg.norm(Om.double()))
    delta = v0 * 10.0 ** 2.5
    pc = api.nys_factor(ctx, Om, -delta * Om, EPS64)
    ref = oracle.nystrom.nystrom(lambda V: -delta * V, Om.reshape(ell, -1).cpu().numpy(), EPS64)
    assert ref["retries"] == 3 and pc.chol_retries == 3
    assert abs(pc.v - ref["v"]) <= 1e-12 * ref["v"]
    assert np.max(np.abs(pc.S_hat.cpu().numpy() - ref["S_hat"])) <= 1e-8 * max(ref["S_hat"][0], 1e-300) + 1e-12


@pytest.mark.parametrize("ell", [64, 200])
def test_not_spd_core_is_reported_on_the_cluster_path(env, ell):
    torch, api, ctx = env
    from paper_2411_08178_gb300._abi import NYS_ENOTSPD, NysError
    Om = torch.from_numpy(gaussian_matrix(32 * 32, ell, 2).reshape(ell, 32, 32)).cuda()
    with pytest.raises(NysError) as e:
        api.nys_factor(ctx, Om, -Om, EPS64)
    assert e.value.code == NYS_ENOTSPD


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("sqrt_shift,mu", [(True, 0.0), (False, 1e-2)])
def test_precond_apply_matches_oracle(env, dt, sqrt_shift, mu):
    torch, api, ctx = env
    n, ell = 48, 16
    h = gaussian_kernel(5, 1.0)
    opo = O.Operator("blur", n, n, kernel=h)
    ref = oracle.nystrom.nystrom(_flat_phi(opo, n, n), gaussian_matrix(n * n, ell, 6), EPS64)
    P = oracle.nystrom.Precond(ref["U"], ref["S_hat"], mu=mu, sqrt_shift=sqrt_shift)
    tdt = torch.float64 if dt == "f64" else torch.float32
    pc = api.Precond(ctx, n * n, ell, tdt).import_factor(ref["U"], ref["S_hat"], mu, sqrt_shift)
    z = gaussian_probe_like((3, n * n), seed=12)
    zg = torch.from_numpy(z).to(tdt).cuda()
    close(api.precond_apply(ctx, pc, zg, inverse=True).cpu(), P.inverse(z), TOL[dt])
    close(api.precond_apply(ctx, pc, zg, inverse=False).cpu(), P.apply(z), TOL[dt])
    # P P^{-1} z = z on the device, in place
    w = api.precond_apply(ctx, pc, zg, inverse=True)
    api.precond_apply(ctx, pc, w, inverse=False, out=w)
    close(w.cpu(), z, TOL[dt])


def test_precond_degenerate_is_reported(env):
    torch, api, ctx = env
    from paper_2411_08178_gb300._abi import NYS_EDEGENERATE, NysError
    U = np.linalg.qr(np.random.default_rng(0).standard_normal((100, 3)))[0].T
    with pytest.raises(NysError) as e:
        api.Precond(ctx, 100, 3, torch.float64).import_factor(U, np.array([2.0, 1.0, 0.0]), 0.0, True)
    assert e.value.code == NYS_EDEGENERATE


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("reg", ["tv", "hs"])
@pytest.mark.parametrize("precond", [False, True])
@pytest.mark.parametrize("shape", [(40, 52), (27, 31)])
def test_prox_dual_matches_oracle(env, dt, reg, precond, shape):
    # (40, 52): the fused dual step (two launches for TV, three for HS);
    # (27, 31): N not a multiple of the vector width, the unfused path
    torch, api, ctx = env
    (n1, n2), ell = shape, 10
    s = phantom(max(n1, n2), 6, 3, "mixed")[:n1, :n2] + 0.05 * gaussian_probe_like((n1, n2), 13)
    lb, n_inner = 0.02, 30
    tdt = torch.float64 if dt == "f64" else torch.float32
    P, pc = oracle.nystrom.Identity(), None
    if precond:
        h = gaussian_kernel(5, 1.0)
        opo = O.Operator("blur", n1, n2, kernel=h)
        ref = oracle.nystrom.nystrom(_flat_phi(opo, n1, n2), gaussian_matrix(n1 * n2, ell, 7), EPS64)
        # without the sqrt heuristic: 9 of the 10 columns get d_i > 0 here
        P = oracle.nystrom.Precond(ref["U"], ref["S_hat"], 0.0, False)
        pc = api.Precond(ctx, n1 * n2, ell, tdt).import_factor(ref["U"], ref["S_hat"], 0.0, False)
        assert pc.ell_active == ell - 1
    x_ref, Q_ref = oracle.prox.prox_dual(s, reg, lb, P, n_inner)
    sg = torch.from_numpy(s).to(tdt).cuda()
    fn = api.prox_tv if reg == "tv" else api.prox_hs
    x, Q = fn(ctx, pc, lb, n_inner, sg)
    tol = TOL[dt] * (10 if dt == "f32" else 1)
    close(x.cpu(), x_ref, tol, 10 * tol)
    close(Q.cpu(), Q_ref, tol * 10, 100 * tol)
    # warm start continues the same sequence of Q (restart of t)
    x2, Q2 = fn(ctx, pc, lb, n_inner, sg, Q=Q)
    x2_ref, _ = oracle.prox.prox_dual(s, reg, lb, P, n_inner, Q0=Q_ref)
    close(x2.cpu(), x2_ref, tol * 10, 100 * tol)


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("reg", ["isotv", "hs2", "hsinf"])
@pytest.mark.parametrize("precond", [False, True])
@pytest.mark.parametrize("shape", [(40, 52), (27, 31)])
def test_prox_mixed_variants_match_oracle(env, dt, reg, precond, shape):
    # isotropic TV, HS_2 and HS_inf through prox_mixed: the fused launches
    # (40 x 52 with P) and the unfused ones (27 x 31, or P = I) against the
    # oracle's dual APG, then a warm start from the returned Q
    torch, api, ctx = env
    (n1, n2), ell = shape, 10
    s = phantom(max(n1, n2), 6, 3, "mixed")[:n1, :n2] + 0.05 * gaussian_probe_like((n1, n2), 13)
    lb, n_inner = 0.02, 30
    tdt = torch.float64 if dt == "f64" else torch.float32
    P, pc = oracle.nystrom.Identity(), None
    if precond:
        h = gaussian_kernel(5, 1.0)
        opo = O.Operator("blur", n1, n2, kernel=h)
        ref = oracle.nystrom.nystrom(_flat_phi(opo, n1, n2), gaussian_matrix(n1 * n2, ell, 7), EPS64)
        P = oracle.nystrom.Precond(ref["U"], ref["S_hat"], 0.0, False)
        pc = api.Precond(ctx, n1 * n2, ell, tdt).import_factor(ref["U"], ref["S_hat"], 0.0, False)
        assert pc.ell_active == ell - 1
    x_ref, Q_ref = oracle.prox.prox_dual(s, reg, lb, P, n_inner)
    sg = torch.from_numpy(s).to(tdt).cuda()
    x, Q = api.prox_mixed(ctx, pc, reg, lb, n_inner, sg)
    tol = TOL[dt] * (10 if dt == "f32" else 1)
    close(x.cpu(), x_ref, tol, 10 * tol)
    close(Q.cpu(), Q_ref, tol * 10, 100 * tol)
    x2, _ = api.prox_mixed(ctx, pc, reg, lb, n_inner, sg, Q=Q)
    x2_ref, _ = oracle.prox.prox_dual(s, reg, lb, P, n_inner, Q0=Q_ref)
    close(x2.cpu(), x2_ref, tol * 10, 100 * tol)


def test_prox_mixed_rejects_wavelet(env):
    torch, api, ctx = env
    from paper_2411_08178_gb300._abi import NYS_EINVAL, NYS_REG_WAVELET, NysError
    s = torch.zeros(8, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(NysError) as e:
        api._prox_dual(lambda *a: api._lib().prox_mixed(a[0], a[1], NYS_REG_WAVELET, *a[2:]), 2, ctx, None,
                       0.1, 3, s)
    assert e.value.code == NYS_EINVAL


@pytest.mark.parametrize("precond", [False, True, "inactive"])
@pytest.mark.parametrize("n_inner", [0, 1, 2, 3, 7])
def test_prox_tv_fused_dual_step_inner_counts(env, precond, n_inner):
    # the TV dual step fused with the L^T after it keeps (R, Q) in two
    # buffers, starts from the caller's Q and writes the last Q back into it:
    # every inner count from 0 up, from a nonzero warm start, against the
    # oracle; "inactive": a factor with no d_i > 0, where P = I exactly
    torch, api, ctx = env
    n1, n2, ell = 40, 52, 10
    s = phantom(max(n1, n2), 6, 3, "mixed")[:n1, :n2] + 0.05 * gaussian_probe_like((n1, n2), 13)
    Q0 = np.clip(np.random.default_rng(4).normal(0.0, 0.6, (2, n1, n2)), -1.0, 1.0)
    lb = 0.02
    P, pc = oracle.nystrom.Identity(), None
    if precond:
        h = gaussian_kernel(5, 1.0)
        opo = O.Operator("blur", n1, n2, kernel=h)
        ref = oracle.nystrom.nystrom(_flat_phi(opo, n1, n2), gaussian_matrix(n1 * n2, ell, 7), EPS64)
        S_hat = ref["S_hat"] if precond is True else np.full(ell, ref["S_hat"][-1])   # all d_i = 0
        P = oracle.nystrom.Precond(ref["U"], S_hat, 0.0, False)
        pc = api.Precond(ctx, n1 * n2, ell, torch.float64).import_factor(ref["U"], S_hat, 0.0, False)
        assert pc.ell_active == (ell - 1 if precond is True else 0)
    x_ref, Q_ref = oracle.prox.prox_dual(s, "tv", lb, P, n_inner, Q0=Q0)
    Qg = torch.from_numpy(Q0).cuda()
    x, Q = api.prox_tv(ctx, pc, lb, n_inner, torch.from_numpy(s).cuda(), Q=Qg)
    close(x.cpu(), x_ref, 1e-12, 1e-11)
    close(Q.cpu(), Q_ref, 1e-12, 1e-11)
    if n_inner == 0:
        assert torch.equal(Q.cpu(), torch.from_numpy(Q0))


@pytest.mark.parametrize("ell,reg", [(16, "tv"), (16, "hs"), (96, "tv")])
def test_prox_fused_bf16_matches_composed(env, ell, reg):
    # the fused dual step with a bf16 U (last-CTA coefficients for
    # ell_active <= 64, two extra passes otherwise) against the same
    # iteration composed from the standalone
    # P^-1 apply and torch stencils, on the same stored U
    torch, api, ctx = env
    n = 64
    h = gaussian_kernel(9, 1.5)
    op = api.Operator(ctx, "blur", n, n, dtype=torch.float32, kernel=h)
    Om, Y = api.nys_sketch(ctx, op, ell, seed=6, store_dtype=torch.bfloat16)
    pc = api.nys_factor(ctx, Om, Y, EPS32, u_dtype=torch.bfloat16)
    pc.setup(0.0, False)
    s = torch.from_numpy(phantom(n, 6, 2, "mixed")).float().cuda()
    lb, n_inner = 0.02, 12
    fn = api.prox_tv if reg == "tv" else api.prox_hs
    x, Q = fn(ctx, pc, lb, n_inner, s)
    # composed reference
    sh = lambda a, di, dj: torch.roll(a, shifts=(-di, -dj), dims=(-2, -1))
    if reg == "tv":
        L = lambda v: torch.stack([v - sh(v, -1, 0), v - sh(v, 0, -1)])
        Lt = lambda q: (q[0] - sh(q[0], 1, 0)) + (q[1] - sh(q[1], 0, 1))
        proj = lambda z: z.clamp(-1.0, 1.0)
        normL2 = 8.0
    else:
        def L(v):
            return torch.stack([sh(v, -1, 0) - 2 * v + sh(v, 1, 0),
                                0.25 * (sh(v, 1, 1) - sh(v, 1, -1) - sh(v, -1, 1) + sh(v, -1, -1)),
                                sh(v, 0, -1) - 2 * v + sh(v, 0, 1)])

        def Lt(q):
            a11 = sh(q[0], -1, 0) - 2 * q[0] + sh(q[0], 1, 0)
            a22 = sh(q[2], 0, -1) - 2 * q[2] + sh(q[2], 0, 1)
            a12 = 0.25 * (sh(q[1], 1, 1) - sh(q[1], 1, -1) - sh(q[1], -1, 1) + sh(q[1], -1, -1))
            return a11 + 2 * a12 + a22

        def proj(z):
            a, b, c = z[0].double(), z[1].double(), z[2].double()
            m, hh = 0.5 * (a + c), 0.5 * (a - c)
            r = torch.sqrt(hh * hh + b * b)
            l1, l2 = (m + r).clamp(-1, 1), (m - r).clamp(-1, 1)
            mp, dp = 0.5 * (l1 + l2), 0.5 * (l1 - l2)
            rs = torch.where(r > 0, r, torch.ones_like(r))
            pa = torch.where(r > 0, mp + dp * hh / rs, mp)
            pb = torch.where(r > 0, dp * b / rs, torch.zeros_like(r))
            pc_ = torch.where(r > 0, mp - dp * hh / rs, mp)
            return torch.stack([pa, pb, pc_]).float()
        normL2 = 32.0
    pinv = lambda z: api.precond_apply(ctx, pc, z.contiguous().reshape(-1), True).reshape(n, n)
    G = 2 if reg == "tv" else 3
    Qp = torch.zeros(G, n, n, device="cuda")
    R = Qp.clone()
    t = 1.0
    for _ in range(n_inner):
        xr = s - lb * pinv(Lt(R))
        Qn = proj(R + L(xr) / (lb * normL2))
        tn = 0.5 * (1.0 + (1.0 + 4.0 * t * t) ** 0.5)
        R = Qn + ((t - 1.0) / tn) * (Qn - Qp)
        Qp, t = Qn, tn
    xr = s - lb * pinv(Lt(Qp))
    assert ell - 2 <= pc.ell_active < ell      # the last column has d = 0 without the sqrt heuristic
    assert rel(x.cpu(), xr.cpu()) < 1e-5
    assert rel(Q.cpu(), Qp.cpu()) < 1e-4


def test_prox_wavelet_matches_oracle(env):
    torch, api, ctx = env
    n, ell = 64, 32
    h = gaussian_kernel(9, 1.5)
    opo = O.Operator("blur", n, n, kernel=h)
    phi = lambda V: O.haar_forward(opo.normal(O.haar_adjoint(V.reshape(-1, n, n), 3)), 3).reshape(V.shape[0], -1)
    ref = oracle.nystrom.nystrom(phi, gaussian_matrix(n * n, ell, 3), EPS64)
    P = oracle.nystrom.Precond(ref["U"], ref["S_hat"])
    pc = api.Precond(ctx, n * n, ell, torch.float64).import_factor(ref["U"], ref["S_hat"], 0.0, True)
    s = O.haar_forward(phantom(n, 8, 1, "mixed"), 3).ravel() + 0.01 * gaussian_probe_like(n * n, 14)
    tau = 0.02
    x_ref, g_ref, it, ok = oracle.prox.prox_wavelet(s, P.Ubar, tau)
    assert ok
    gamma = torch.zeros(ell, dtype=torch.float64, device="cuda")
    x, info = api.prox_wavelet(ctx, pc, tau, torch.from_numpy(s).cuda(), gamma=gamma)
    assert info["converged"]
    assert rel(x.cpu(), x_ref) < 1e-10
    assert rel(gamma.cpu(), g_ref) < 1e-8
    # P = I: soft threshold
    x0, _ = api.prox_wavelet(ctx, None, tau, torch.from_numpy(s).cuda())
    assert rel(x0.cpu(), oracle.prox.soft_threshold(s, tau)) < 1e-15
