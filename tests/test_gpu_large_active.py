"""GPU parity of the large-active-set path against the float64 oracle.

With more than 64 columns of U active (d_i > 0), P^{-1} and the P-metric prox
take different kernels than the small-set tests exercise: the partial sums of
U^T g are reduced by a column pass and c = M w by a row pass over many CTAs
(instead of the last CTA of the partial-sum pass), the pixel chunks are half
as long, and the x pass streams two columns x two 16-byte vectors per lane.
The CT sketch (ell = 400, every column active) runs exactly this path.

Each case imports one oracle factor (a 9 x 9 Gaussian blur at 128 x 128,
ell = 200, without the square-root heuristic: 199 active columns) into the
library and compares P^{-1}, P, the TV and HS proxes and ten WAPG iterations.
A bf16 U is compared against the oracle's definitions evaluated on the same
bf16-rounded U: P z = z + U diag(d) U^T z holds for any U, and P^{-1} is the
exact inverse of that P (Woodbury identity, checked here against P itself).
"""
import numpy as np
import pytest

import oracle
from oracle import operators as O
from oracle.philox import gaussian_matrix
from workloads import gaussian_kernel, gaussian_probe_like, phantom
from tests.gpu_util import TOL, close, maxrel, rel, require_gpu

pytestmark = pytest.mark.gpu
N1 = 128
ELL = 200
EPS64 = 2.0 ** -52


@pytest.fixture(scope="module")
def env():
    torch, api = require_gpu()
    return torch, api, api.Context(0)


@pytest.fixture(scope="module")
def factor():
    h = gaussian_kernel(9, 1.5)
    opo = O.Operator("blur", N1, N1, kernel=h)
    phi = lambda V: opo.normal(V.reshape(-1, N1, N1)).reshape(V.shape[0], -1)
    ref = oracle.nystrom.nystrom(phi, gaussian_matrix(N1 * N1, ELL, 7), EPS64)
    return opo, h, ref


class WoodburyInverse:
    """P = I + U^T diag(d) U for rows U (any U, not only orthonormal) and its
    exact inverse I - V (I + V^T V)^{-1} V^T, V = U^T diag(sqrt d)."""

    def __init__(self, U, d):
        self.U, self.d = U, d
        V = U.T * np.sqrt(d)
        self.V = V
        self.core = np.linalg.inv(np.eye(U.shape[0]) + V.T @ V)

    def apply(self, z):
        z = np.asarray(z, dtype=np.float64)
        flat = z.reshape(z.shape[:-2] + (-1,)) if z.ndim >= 2 and z.shape[-1] != self.U.shape[1] else z
        w = flat @ self.U.T
        return (flat + (w * self.d) @ self.U).reshape(z.shape)

    def inverse(self, z):
        z = np.asarray(z, dtype=np.float64)
        flat = z.reshape(z.shape[:-2] + (-1,)) if z.ndim >= 2 and z.shape[-1] != self.U.shape[1] else z
        return (flat - ((flat @ self.V) @ self.core) @ self.V.T).reshape(z.shape)


def _oracle_precond(torch, ref, ud):
    """The oracle preconditioner on the U the library will hold."""
    d = oracle.nystrom.precond_weights(ref["S_hat"], 0.0, False)
    if ud == "bf16":
        Ub = torch.from_numpy(ref["U"]).to(torch.bfloat16).double().numpy()
        W = WoodburyInverse(Ub, d)
        z = gaussian_probe_like((2, N1 * N1), seed=40)
        assert rel(W.apply(W.inverse(z)), z) < 1e-12       # the inverse is P's
        return W
    return oracle.nystrom.Precond(ref["U"], ref["S_hat"], 0.0, False)


def _library_precond(torch, api, ctx, ref, ud):
    tdt = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16}[ud]
    pc = api.Precond(ctx, N1 * N1, ELL, tdt).import_factor(ref["U"], ref["S_hat"], 0.0, False)
    assert pc.ell_active == ELL - 1 > 64
    return pc


@pytest.mark.parametrize("ud", ["f32", "f64", "bf16"])
def test_precond_large_active_matches_oracle(env, factor, ud):
    torch, api, ctx = env
    _, _, ref = factor
    P = _oracle_precond(torch, ref, ud)
    pc = _library_precond(torch, api, ctx, ref, ud)
    zdt = torch.float64 if ud == "f64" else torch.float32
    tol = TOL["f64"] * 10 if ud == "f64" else TOL["f32"]
    z = gaussian_probe_like((3, N1 * N1), seed=41)
    zg = torch.from_numpy(z).to(zdt).cuda()
    close(api.precond_apply(ctx, pc, zg, inverse=True), P.inverse(z), tol)
    close(api.precond_apply(ctx, pc, zg, inverse=False), P.apply(z), tol)
    w = api.precond_apply(ctx, pc, zg, inverse=True)
    api.precond_apply(ctx, pc, w, inverse=False, out=w)
    close(w, z, tol)


@pytest.mark.parametrize("ud", ["f32", "f64", "bf16"])
@pytest.mark.parametrize("reg", ["tv", "hs"])
def test_prox_large_active_matches_oracle(env, factor, ud, reg):
    torch, api, ctx = env
    _, _, ref = factor
    P = _oracle_precond(torch, ref, ud)
    pc = _library_precond(torch, api, ctx, ref, ud)
    s = phantom(N1, 6, 3, "mixed") + 0.05 * gaussian_probe_like((N1, N1), 13)
    lb, n_inner = 0.02, 30
    x_ref, Q_ref = oracle.prox.prox_dual(s, reg, lb, P, n_inner)
    tdt = torch.float64 if ud == "f64" else torch.float32
    fn = api.prox_tv if reg == "tv" else api.prox_hs
    x, Q = fn(ctx, pc, lb, n_inner, torch.from_numpy(s).to(tdt).cuda())
    tol = 1e-11 if ud == "f64" else 1e-4
    close(x, x_ref, tol, 10 * tol)
    close(Q, Q_ref, 10 * tol, 100 * tol)
    x2, _ = fn(ctx, pc, lb, n_inner, torch.from_numpy(s).to(tdt).cuda(), Q=Q)
    x2_ref, _ = oracle.prox.prox_dual(s, reg, lb, P, n_inner, Q0=Q_ref)
    close(x2, x2_ref, 10 * tol, 100 * tol)


@pytest.mark.parametrize("ud", ["f32", "f64"])
def test_wapg_large_active_matches_oracle(env, factor, ud):
    # ten preconditioned iterations of TV deblurring with the oracle's factor
    # and step size on both sides
    torch, api, ctx = env
    opo, h, ref = factor
    P = _oracle_precond(torch, ref, ud)
    pc = _library_precond(torch, api, ctx, ref, ud)
    x_true = phantom(N1, 12, 5, "ellipse")
    y = opo.apply(x_true) + np.random.default_rng(6).normal(0.0, 0.01, (N1, N1))
    prob = oracle.wapg.Problem(opo, y, 2e-3, "tv")
    alpha = 1.0 / oracle.wapg.power_lipschitz(prob, P)
    x_ref = oracle.wapg.wapg(prob, alpha, 10, precond=P, n_inner=10)["x"]
    tdt = torch.float64 if ud == "f64" else torch.float32
    op = api.Operator(ctx, "blur", N1, N1, dtype=tdt, kernel=h)
    sol = api.Solver(ctx, op, torch.from_numpy(y).to(tdt).cuda(), "tv", 2e-3, pc=pc, alpha=alpha, n_inner=10)
    sol.step(10)
    x = sol.x()
    tol = 1e-10 if ud == "f64" else 1e-4
    close(x, x_ref, tol, 10 * tol)
    assert maxrel(x, x_ref) < 10 * tol
