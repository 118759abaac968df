"""The sharding entry points on one GPU, through the C ABI: a column slice of
the sketch equals the same columns of the whole sketch; the factor built from
row slices (partial Grams summed on the host, as an all-reduce would) equals
nys_factor; the split P^{-1} apply (partial sums of each row slice added on
the host) equals precond_apply.  The ranks are run one after the other on
the same device: none of their kernels waits for another's."""
import numpy as np
import pytest

from workloads import gaussian_kernel, gaussian_probe_like
from tests.gpu_util import close, rel, require_gpu

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -23


@pytest.fixture(scope="module")
def env():
    torch, api = require_gpu()
    return torch, api, api.Context(0)


@pytest.mark.parametrize("sd", ["f32", "bf16"])
def test_sketch_columns_equal_the_whole_sketch(env, sd):
    torch, api, ctx = env
    n, ell = 40, 12
    op = api.Operator(ctx, "blur", n, n, dtype=torch.float32, kernel=gaussian_kernel(7, 1.3))
    tsd = torch.bfloat16 if sd == "bf16" else torch.float32
    Om, Y = api.nys_sketch(ctx, op, ell, seed=17, store_dtype=tsd)
    for j0, j1 in [(0, 5), (5, 12), (3, 4), (11, 12)]:
        Oc, Yc = api.nys_sketch_cols(ctx, op, ell, j0, j1, seed=17, store_dtype=tsd)
        assert torch.equal(Oc, Om[j0:j1]) and torch.equal(Yc, Y[j0:j1])


def _row_slices(N, parts):
    from paper_2411_08178_gb300.sharded import split
    return split(N, parts, 8)


@pytest.mark.parametrize("sd,parts", [("f32", 2), ("bf16", 3)])
def test_factor_from_row_slices_equals_nys_factor(env, sd, parts):
    torch, api, ctx = env
    n, ell = 64, 96
    op = api.Operator(ctx, "blur", n, n, dtype=torch.float32, kernel=gaussian_kernel(9, 1.5))
    tsd = torch.bfloat16 if sd == "bf16" else torch.float32
    Om, Y = api.nys_sketch(ctx, op, ell, seed=19, store_dtype=tsd)
    pc = api.nys_factor(ctx, Om, Y, EPS32, u_dtype=tsd)
    O2, Y2 = Om.reshape(ell, -1), Y.reshape(ell, -1)
    rows = _row_slices(n * n, parts)
    G2 = torch.zeros((2 * ell, 2 * ell), dtype=torch.float64, device="cuda")
    for a, b in rows:
        Oa, Ya = O2[:, a:b].contiguous(), Y2[:, a:b].contiguous()
        G2[:ell, :ell] += api.nys_gram(ctx, Oa, Oa)
        G2[:ell, ell:] += api.nys_gram(ctx, Oa, Ya)
        G2[ell:, ell:] += api.nys_gram(ctx, Ya, Ya)
    W, S, v, _ = api.nys_factor_gram(ctx, G2, ell, EPS32)
    tol = 1e-4 if sd == "f32" else 3e-2
    assert abs(v - pc.v) <= 1e-6 * pc.v
    assert np.max(np.abs(S.cpu().numpy() - pc.S_hat.cpu().numpy())) <= tol * pc.S_hat[0].item()
    U = torch.cat([api.nys_tall_gemm(ctx, Y2[:, a:b].contiguous(), O2[:, a:b].contiguous(), v, W, out_dtype=tsd)
                   for a, b in rows], dim=1).double()
    Z = torch.from_numpy(gaussian_probe_like((3, n * n), 5)).cuda()
    Ur = pc.U.double()
    lhs = ((Z @ U.T) * S) @ U
    ref = ((Z @ Ur.T) * pc.S_hat) @ Ur
    assert rel(lhs, ref) < tol


@pytest.mark.parametrize("ud", ["f32", "bf16", "f64"])
def test_split_precond_apply_equals_precond_apply(env, ud):
    torch, api, ctx = env
    n, ell = 64, 80
    dt = torch.float64 if ud == "f64" else torch.float32
    tud = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}[ud]
    op = api.Operator(ctx, "blur", n, n, dtype=dt, kernel=gaussian_kernel(9, 1.5))
    Om, Y = api.nys_sketch(ctx, op, ell, seed=23, store_dtype=tud)
    pc = api.nys_factor(ctx, Om, Y, 2.0 ** -52 if ud == "f64" else EPS32, u_dtype=tud)
    pc.setup(0.0, False)                                   # every column but the last active
    U2 = pc.U.reshape(ell, -1)
    rows = _row_slices(n * n, 2)
    K = sum(api.nys_gram(ctx, U2[:, a:b].contiguous(), U2[:, a:b].contiguous()) for a, b in rows)
    parts = [api.Precond(ctx, b - a, ell, tud).import_gram(U2[:, a:b], pc.S_hat, K, 0.0, False) for a, b in rows]
    z = torch.from_numpy(gaussian_probe_like((2, n * n), 29)).to(dt).cuda()
    zs = [z[:, a:b].contiguous() for a, b in rows]
    w = sum(api.precond_partial(ctx, p, zz) for p, zz in zip(parts, zs))
    tol = 1e-12 if ud == "f64" else 1e-5
    for inverse in (True, False):
        out = torch.cat([api.precond_finish(ctx, p, w, zz, inverse) for p, zz in zip(parts, zs)], dim=1)
        close(out, api.precond_apply(ctx, pc, z, inverse=inverse), tol)
