"""Error of the reduced-precision sketch path against the float64 oracle.

The GPU builds U and S_hat from bf16 (the benchmark configuration: Omega, Y
and U stored in bf16, tcgen05 Gram and tall GEMM with float32 accumulation,
float64 shift, Cholesky and core algebra, float32 Jacobi with float64
Rayleigh quotients) and from float32 storage, starting from the same Omega
(the shared Philox definition) as the float64 oracle's Algorithm 1 with the
same machine accuracy eps = 2^-23.  Reported (printed as one JSON line) and
gated loosely:
  * the low-rank operator: ||U S U^T Z - U0 S0 U0^T Z||_F / ||U0 S0 U0^T Z||_F
    on 8 random probe vectors Z,
  * the largest relative error among the top 10 eigenvalues and of the last,
  * the final image after 60 TV-regularised WAPG iterations, each side with
    its own P and its own power-iteration step size.
Workload: the 25 x 25 sigma 4 deblurring recipe at 192 x 192, ell = 96.
"""
import json

import numpy as np
import pytest

import oracle
import workloads as WL
from oracle import operators as O
from oracle.philox import gaussian_matrix
from tests.gpu_util import rel, require_gpu

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -23


@pytest.fixture(scope="module")
def setup():
    torch, api = require_gpu()
    ctx = api.Context(0)
    w = WL.scaled(WL.DEBLUR512, 192, ell=96)
    n, ell = w.n, w.ell
    h = WL.blur_kernel_for(w)
    opo = O.Operator("blur", n, n, kernel=h)
    x_true = WL.ground_truth(w)
    y = WL.degrade(w, opo.apply(x_true))
    prob = oracle.wapg.Problem(opo, y, w.lam, "tv")
    phi = lambda V: opo.normal(V.reshape(-1, n, n)).reshape(V.shape[0], -1)
    ref = oracle.nystrom.nystrom(phi, gaussian_matrix(n * n, ell, w.seed_omega), EPS32)
    P0 = oracle.nystrom.Precond(ref["U"], ref["S_hat"])
    a0 = 1.0 / oracle.wapg.power_lipschitz(prob, P0)
    K = 60
    x0 = oracle.wapg.wapg(prob, a0, K, precond=P0, n_inner=w.n_inner)["x"]
    return torch, api, ctx, w, h, y, ref, x0, K


@pytest.mark.parametrize("store", ["bf16", "f32"])
def test_reduced_precision_factor_and_image_vs_float64(setup, store):
    torch, api, ctx, w, h, y, ref, x0, K = setup
    n, ell, N = w.n, w.ell, w.n * w.n
    sd = torch.bfloat16 if store == "bf16" else torch.float32
    op = api.Operator(ctx, "blur", n, n, dtype=torch.float32, kernel=h)
    Om, Y = api.nys_sketch(ctx, op, ell, w.seed_omega, store_dtype=sd)
    pc = api.Precond(ctx, N, ell, sd)
    api.nys_factor(ctx, Om, Y, EPS32, pc=pc)
    ctx.sync()
    U = pc.U.double().cpu().numpy().reshape(ell, N)
    S = pc.S_hat.cpu().numpy()
    U0, S0 = ref["U"].reshape(ell, N), ref["S_hat"]
    Z = np.random.default_rng(5).standard_normal((N, 8))
    A0 = U0.T @ (S0[:, None] * (U0 @ Z))
    A1 = U.T @ (S[:, None] * (U @ Z))
    e_op = float(np.linalg.norm(A1 - A0) / np.linalg.norm(A0))
    e_top = float(np.max(np.abs(S[:10] - S0[:10]) / S0[:10]))
    e_last = float(abs(S[-1] - S0[-1]) / S0[-1])
    sol = api.Solver(ctx, op, torch.from_numpy(y).float().cuda(), "tv", w.lam, pc=pc, n_inner=w.n_inner)
    sol.step(K)
    e_img = rel(sol.x().cpu(), x0)
    rep = {"store": store, "workload": f"deblur {n}x{n} 25x25 sigma 4, ell {ell}", "lowrank_op_rel": e_op,
           "s_hat_top10_max_rel": e_top, "s_hat_last_rel": e_last, "v_gpu": pc.v, "v_oracle": ref["v"],
           "image_rel_after_60_iters": e_img, "active_columns": pc.ell_active}
    print("PRECISION " + json.dumps(rep))
    lim = {"bf16": (5e-2, 2e-2, 1e-2), "f32": (1e-3, 1e-4, 1e-3)}[store]
    assert e_op < lim[0] and e_top < lim[1] and e_img < lim[2], rep
