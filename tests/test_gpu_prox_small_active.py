"""GPU parity of the one-launch P-metric TV dual step (up to 64 active
columns): each launch stages x = s - lb (g - U c) of the previous step on its
1024-pixel chunk and one image row either side, then runs the fused dual
update, L^T and the U^T g partial sums.

The shapes cover a last chunk shorter than 1024 pixels, a chunk whose rows
wrap around the image (first and last chunks), images too small for the
staged path (N < 1024 + 2 n2: the two-launch step), widths that are not a
multiple of the 16-byte vector (two-launch step), the first and last dual
step (n_inner = 1, 2, 9) and a warm start.  U is a seeded Gaussian matrix;
the oracle is P = I + U^T diag(d) U on the U the library holds and its exact
inverse, inside the oracle's dual APG.
"""
import numpy as np
import pytest

import oracle
from workloads import gaussian_probe_like, phantom
from tests.gpu_util import close, maxrel, require_gpu
from tests.test_gpu_large_active import WoodburyInverse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, api = require_gpu()
    return torch, api, api.Context(0)


CASES = [
    (33, 64, 30, "bf16"),    # staged; chunks 1024, 1024, 64
    (20, 64, 12, "f32"),     # staged; the last chunk's rows wrap to row 0
    (48, 96, 65, "f32"),     # 64 active columns (the most the one-launch step takes)
    (12, 96, 20, "f32"),     # N < 1024 + 2 n2: two launches per step
    (40, 52, 17, "bf16"),    # 52 not a multiple of 8: two launches per step
    (64, 64, 40, "f64"),     # float64 U and iterates, staged
]


@pytest.mark.parametrize("n1,n2,ell,ud", CASES)
@pytest.mark.parametrize("n_inner", [1, 2, 9])
def test_prox_tv_small_active_matches_oracle(env, n1, n2, ell, ud, n_inner):
    torch, api, ctx = env
    N = n1 * n2
    rng = np.random.default_rng(n1 * 31 + ell)
    U = rng.standard_normal((ell, N)) / np.sqrt(N)
    S_hat = np.sort(rng.uniform(1.0, 30.0, ell))[::-1].copy()
    tdt = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16}[ud]
    Ul = torch.from_numpy(U).to(tdt).double().numpy()
    P = WoodburyInverse(Ul, oracle.nystrom.precond_weights(S_hat, 0.0, False))
    pc = api.Precond(ctx, N, ell, tdt).import_factor(U, S_hat, 0.0, False)
    assert pc.ell_active == ell - 1 <= 64
    s = phantom(max(n1, n2), 5, 2, "mixed")[:n1, :n2] + 0.05 * gaussian_probe_like((n1, n2), 21)
    idt = torch.float64 if ud == "f64" else torch.float32
    lb = 0.03
    x_ref, Q_ref = oracle.prox.prox_dual(s, "tv", lb, P, n_inner)
    x, Q = api.prox_tv(ctx, pc, lb, n_inner, torch.from_numpy(s).to(idt).cuda())
    tol = 1e-11 if ud == "f64" else 1e-4
    close(x, x_ref, tol, 10 * tol)
    close(Q, Q_ref, 10 * tol, 100 * tol)
    x2, _ = api.prox_tv(ctx, pc, lb, n_inner, torch.from_numpy(s).to(idt).cuda(), Q=Q)
    x2_ref, _ = oracle.prox.prox_dual(s, "tv", lb, P, n_inner, Q0=Q_ref)
    close(x2, x2_ref, 10 * tol, 100 * tol)
    assert maxrel(x2, x2_ref) < 100 * tol
