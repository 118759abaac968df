"""GPU parity of Algorithm 2 (IRM with preconditioned CG and the on-the-fly
Nystrom preconditioner) against the float64 oracle, and its properties in
float32 with a bf16 sketch."""
import numpy as np
import pytest

from oracle import irm as IR
from oracle import operators as O
from workloads import gaussian_kernel, phantom
from tests.gpu_util import rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, api = require_gpu()
    return torch, api, api.Context(0)


def _problem(n, k, seed, sigma=1.2):
    rng = np.random.default_rng(seed)
    h = gaussian_kernel(k, sigma)
    op = O.Operator("blur", n, n, kernel=h)
    x_true = phantom(n, 5, seed, "mixed")
    y = op.apply(x_true) + rng.normal(0, 0.01, (n, n))
    m = rng.uniform(size=(n, n))
    y = np.where(m < 0.05, 1.0, np.where(m > 0.95, 0.0, y))        # salt and pepper
    return h, op, y, x_true


@pytest.mark.parametrize("p,q,ell", [(1.0, 1.0, 0), (1.0, 1.0, 12), (0.8, 0.5, 12)])
def test_irm_matches_oracle_f64(env, p, q, ell):
    torch, api, ctx = env
    n, lam, eps, outer = 16, 0.02, 1e-4, 3
    h, opo, y, _ = _problem(n, 5, 1)
    x_ref, hist = IR.irm(opo, y, lam, p, q, eps, outer, ell=ell, seed=3, cg_tol=1e-11, cg_max=3000)
    op = api.Operator(ctx, "blur", n, n, dtype=torch.float64, kernel=h)
    irm = api.IRM(ctx, op, torch.from_numpy(y).cuda(), p, q, lam, eps, ell=ell, seed=3, cg_tol=1e-11, cg_max=3000)
    for k in range(outer):
        info = irm.step()
        assert abs(info["cg_iters"] - hist[k]["cg_iters"]) <= 2, (k, info, hist[k])
        assert info["residual"] <= 1e-11
    assert rel(irm.x().cpu(), x_ref) < 1e-8


def test_irm_f32_bf16_sketch_decreases_objective_and_saves_cg(env):
    torch, api, ctx = env
    n, lam, eps, p, q = 64, 0.01, 1e-3, 1.0, 1.0
    h, opo, y, _ = _problem(n, 9, 2, sigma=2.0)
    op = api.Operator(ctx, "blur", n, n, dtype=torch.float32, kernel=h)
    yt = torch.from_numpy(y).float().cuda()
    runs = {}
    for ell in (0, 48):
        irm = api.IRM(ctx, op, yt, p, q, lam, eps, ell=ell, store_dtype=torch.bfloat16, seed=5, cg_tol=1e-4,
                      cg_max=8000)
        F = [IR.smoothed_objective(opo, y, np.zeros((n, n)), lam, p, q, eps)]
        its = []
        for _ in range(4):
            info = irm.step()
            assert info["residual"] <= 1e-4
            its.append(info["cg_iters"])
            F.append(IR.smoothed_objective(opo, y, irm.x().double().cpu().numpy(), lam, p, q, eps))
        assert all(b <= a * (1 + 1e-6) for a, b in zip(F, F[1:])), (ell, F)
        runs[ell] = its
        irm.close()
    assert sum(runs[48]) < sum(runs[0]), runs


def test_irm_rejects_bad_arguments(env):
    torch, api, ctx = env
    from paper_2411_08178_gb300._abi import NYS_EINVAL, NysError
    op = api.Operator(ctx, "blur", 8, 8, dtype=torch.float32, kernel=gaussian_kernel(3, 1.0))
    y = torch.zeros(8, 8, device="cuda")
    for kw in (dict(p=0.0), dict(p=2.5), dict(eps=0.0), dict(ell=100)):
        args = dict(p=1.0, q=1.0, lam=0.1, eps=1e-4)
        args.update(kw)
        ell = args.pop("ell", 0)
        with pytest.raises(NysError) as e:
            api.IRM(ctx, op, y, args["p"], args["q"], args["lam"], args["eps"], ell=ell)
        assert e.value.code == NYS_EINVAL
