"""The exact early stop of the anisotropic-TV dual iteration: with it on, the
prox and the solver give results bit-identical to running every dual step,
on each path of the prox (P = I; a low-rank P with at most 64 active columns,
one launch per dual step; more than 64, four launches per step) and in
float32 (float32 and bf16 U) and float64.  A tiny prox weight saturates the
dual within a few steps, so there the stop must also skip steps."""
import numpy as np
import pytest

from workloads import gaussian_kernel, gaussian_probe_like, phantom
from tests.gpu_util import close, require_gpu

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -23


@pytest.fixture(scope="module")
def env():
    torch, api = require_gpu()
    return torch, api, api.Context(0)


def _orthonormal(N, ell, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((N, ell)))
    return q.T.copy()


def _run(torch, api, ctx, pc, lb, n_inner, s, Q0, on):
    ctx.set_dual_stop(on)
    before = ctx.dual_steps_skipped()
    x, Q = api.prox_tv(ctx, pc, lb, n_inner, s, Q=Q0.clone())
    torch.cuda.synchronize()
    return x.clone(), Q.clone(), ctx.dual_steps_skipped() - before


# (active columns, U dtype, data dtype): P = I, <= 64 active (one launch per
# dual step), > 64 active (four launches per step)
CASES = [(0, None, "f32"), (0, None, "f64"), (10, "f32", "f32"), (10, "bf16", "f32"), (10, "f64", "f64"),
         (96, "f32", "f32"), (96, "bf16", "f32"), (96, "f64", "f64")]


@pytest.mark.parametrize("lb,saturates", [(1e-6, True), (0.02, False)])
@pytest.mark.parametrize("ell,udt,dt", CASES)
def test_dual_stop_is_bit_identical(env, ell, udt, dt, lb, saturates):
    torch, api, ctx = env
    n = 64
    tdt = torch.float64 if dt == "f64" else torch.float32
    pc = None
    if ell:
        ud = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}[udt]
        S = np.linspace(2.0, 1.0, ell)
        # without the square-root heuristic: ell - 1 columns with d_i > 0
        pc = api.Precond(ctx, n * n, ell, ud).import_factor(_orthonormal(n * n, ell, 3), S, 0.0, False)
        assert pc.ell_active == ell - 1
    s = torch.from_numpy(phantom(n, 6, 3, "mixed") + 0.05 * gaussian_probe_like((n, n), 9)).to(tdt).cuda()
    Q0 = torch.zeros((2, n, n), dtype=tdt, device="cuda")
    try:
        x_off, Q_off, sk_off = _run(torch, api, ctx, pc, lb, 20, s, Q0, False)
        x_on, Q_on, sk_on = _run(torch, api, ctx, pc, lb, 20, s, Q0, True)
    finally:
        ctx.set_dual_stop(True)
    assert sk_off == 0
    assert torch.equal(x_on, x_off) and torch.equal(Q_on, Q_off)
    if saturates:
        assert sk_on > 0
    # a warm start from the returned Q continues at the fixed point
    if saturates:
        x2, Q2, sk2 = _run(torch, api, ctx, pc, lb, 20, s, Q_on, True)
        assert sk2 >= 17 and torch.equal(Q2, Q_on)
        close(x2.cpu(), x_on.cpu(), 1e-6, 1e-5)


@pytest.mark.parametrize("precond", [False, True])
def test_dual_stop_solver_bit_identical(env, precond):
    # 40 WAPG iterations of a TV deblurring problem whose prox weight
    # alpha lambda is small (1e-6 here, alpha about 1; on the 512^2 CT
    # workload alpha is about 4e-5 and lambda 2e-4), so that the dual
    # saturates: the iterate with the stop on equals the one without, and
    # steps were skipped
    torch, api, ctx = env
    n, ell = 64, 24
    h = gaussian_kernel(9, 1.5)
    op = api.Operator(ctx, "blur", n, n, dtype=torch.float32, kernel=h)
    x_true = torch.from_numpy(phantom(n, 6, 5, "mixed")).float().cuda()
    y = api.op_apply(op, x_true.reshape(1, n, n)).reshape(n, n)
    y = y + 0.01 * torch.from_numpy(gaussian_probe_like((n, n), 2)).float().cuda()
    pc = None
    if precond:
        Om, Y = api.nys_sketch(ctx, op, ell, seed=8, store_dtype=torch.bfloat16)
        pc = api.nys_factor(ctx, Om, Y, EPS32, u_dtype=torch.bfloat16)
    xs, skips = [], []
    try:
        for on in (False, True):
            ctx.set_dual_stop(on)
            before = ctx.dual_steps_skipped()
            sol = api.Solver(ctx, op, y, "tv", 1e-6, pc=pc, n_inner=20)
            sol.step(40)
            xs.append(sol.x().clone())
            skips.append(ctx.dual_steps_skipped() - before)
            sol.close()
    finally:
        ctx.set_dual_stop(True)
    assert skips[0] == 0 and skips[1] > 0
    assert torch.equal(xs[0], xs[1])


@pytest.mark.parametrize("reg", ["isotv", "hs", "hs2", "hsinf"])
@pytest.mark.parametrize("ell,udt,dt", [(0, None, "f32"), (0, None, "f64"), (10, "f32", "f32"), (96, "f32", "f32"),
                                        (96, "f64", "f64")])
def test_dual_stop_mixed_norms_bit_identical(env, reg, ell, udt, dt):
    # the unfused dual steps (L^T, the P^{-1} passes, then the dual update):
    # stop on and off agree bit for bit; a prox weight small enough to
    # saturate the dual gives the stop something to skip
    torch, api, ctx = env
    n, lb = 64, 1e-6
    G = 2 if reg == "isotv" else 3
    tdt = torch.float64 if dt == "f64" else torch.float32
    pc = None
    if ell:
        ud = {"f32": torch.float32, "f64": torch.float64}[udt]
        pc = api.Precond(ctx, n * n, ell, ud).import_factor(_orthonormal(n * n, ell, 3), np.linspace(2.0, 1.0, ell),
                                                            0.0, False)
    s = torch.from_numpy(phantom(n, 6, 3, "mixed") + 0.05 * gaussian_probe_like((n, n), 9)).to(tdt).cuda()
    Q0 = torch.zeros((G, n, n), dtype=tdt, device="cuda")
    out = {}
    try:
        for on in (False, True):
            ctx.set_dual_stop(on)
            before = ctx.dual_steps_skipped()
            x, Q = api.prox_mixed(ctx, pc, reg, lb, 20, s, Q=Q0.clone())
            torch.cuda.synchronize()
            out[on] = (x.clone(), Q.clone(), ctx.dual_steps_skipped() - before)
    finally:
        ctx.set_dual_stop(True)
    print(f"{reg} active {max(ell - 1, 0)} {dt}: {out[True][2]} of 20 dual steps skipped")
    assert out[False][2] == 0
    assert torch.equal(out[True][0], out[False][0]) and torch.equal(out[True][1], out[False][1])
