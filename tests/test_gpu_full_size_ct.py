"""The 512 x 512 parallel-beam CT workload (720 angles, 736 bins, TV,
ell = 400, bf16 sketch) in the launch configuration bench.py times.

Algorithm 1 at full size is checked through properties that hold at any
size (the oracle's QR + SVD of a 262144 x 400 matrix is not the point here):
S_hat descending and non-negative, U^T U = I to the bf16 storage error, and
B B^T Omega = Y_v on sampled sketch columns, i.e. U (S_hat + v) U^T Omega =
Y + v Omega.

The P-metric TV prox on that factor (every column active, the large-set
kernels with the L2-resident leading columns, n_inner = 20) is compared with
the oracle's dual APG element by element: P = I + U^T diag(d) U on the U the
library holds (bf16) and its exact inverse by the Woodbury identity, d from
the library's S_hat with the square-root heuristic.
"""
import numpy as np
import pytest

import oracle
import workloads as WL
from workloads import gaussian_probe_like
from tests.gpu_util import close, maxrel, rel, require_gpu
from tests.test_gpu_large_active import WoodburyInverse

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -23


@pytest.fixture(scope="module")
def ct_factor():
    torch, api = require_gpu()
    ctx = api.Context(0)
    w = WL.PRESETS["ct512_parallel_tv_f32"]
    op = api.Operator(ctx, "radon", w.n, w.n, dtype=torch.float32, n_angles=w.n_angles, n_bins=w.n_bins)
    Om, Y = api.nys_sketch(ctx, op, w.ell, w.seed_omega, store_dtype=torch.bfloat16)
    pc = api.nys_factor(ctx, Om, Y, EPS32, u_dtype=torch.bfloat16)
    return torch, api, ctx, w, Om, Y, pc


def test_ct_factor_full_size_properties(ct_factor):
    torch, api, ctx, w, Om, Y, pc = ct_factor
    U = pc.U.double().reshape(w.ell, -1)
    S = pc.S_hat
    assert torch.all(S[:-1] >= S[1:]) and S[-1] >= 0
    assert pc.ell_active == w.ell
    G = U @ U.T
    assert torch.max(torch.abs(G - torch.eye(w.ell, dtype=torch.float64, device=G.device))).item() < 2e-2
    cols = [0, 13, 199, 399]
    Oc = Om.reshape(w.ell, -1)[cols].double()
    Yc = Y.reshape(w.ell, -1)[cols].double()
    lhs = ((Oc @ U.T) * (S + pc.v)) @ U
    rhs = Yc + pc.v * Oc
    assert rel(lhs.cpu(), rhs.cpu()) < 3e-2


def test_ct_prox_full_size_matches_oracle(ct_factor):
    torch, api, ctx, w, Om, Y, pc = ct_factor
    Ub = pc.U.reshape(w.ell, -1).double().cpu().numpy()   # the bf16 values the kernels read
    S = pc.S_hat.cpu().numpy()
    P = WoodburyInverse(Ub, oracle.nystrom.precond_weights(S, 0.0, True))
    s = WL.ground_truth(w) + 0.05 * gaussian_probe_like((w.n, w.n), 31)
    lb, n_inner = 0.5, 20
    x_ref, Q_ref = oracle.prox.prox_dual(s, "tv", lb, P, n_inner)
    x, Q = api.prox_tv(ctx, pc, lb, n_inner, torch.from_numpy(s).float().cuda())
    close(x, x_ref, 1e-4, 1e-3)
    close(Q, Q_ref, 1e-3, 1e-2)
    # the standalone P^{-1} and P on the same factor, element by element
    z = gaussian_probe_like((w.n * w.n,), 32)
    zg = torch.from_numpy(z).float().cuda()
    close(api.precond_apply(ctx, pc, zg, inverse=True), P.inverse(z), 1e-5, 1e-4)
    close(api.precond_apply(ctx, pc, zg, inverse=False), P.apply(z), 1e-5, 1e-4)
    assert maxrel(x, x_ref) < 1e-3
