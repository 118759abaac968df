"""The sharded sketch and factor (paper_2411_08178_gb300/sharded.py) on CPU with
two and three gloo ranks.

The exchange pattern (column slices of the sketch, the all-to-all into pixel
slices, the all-reduced Grams, the per-rank rows of U, the split P^{-1}) is
the product code; the local steps run through a numpy stand-in of the
library calls defined here, so that the ranks need no GPU.  The assembled
factor must equal the oracle's Algorithm 1 on the whole problem.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N1, ELL, SEED, EPS = 24, 20, 5, 2.0 ** -52


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class NumpyBackend:
    """The library's local steps restated in numpy (float64), for CPU ranks."""

    def __init__(self, n1):
        from oracle import operators as O
        from workloads import gaussian_kernel
        self.n1 = n1
        self.op = O.Operator("blur", n1, n1, kernel=gaussian_kernel(5, 1.2))

    def sketch_cols(self, ell, j0, j1, seed):
        from oracle.philox import gaussian_matrix
        Om = gaussian_matrix(self.n1 * self.n1, ell, seed)[j0:j1]
        Y = self.op.normal(Om.reshape(-1, self.n1, self.n1)).reshape(j1 - j0, -1)
        return torch.from_numpy(Om), torch.from_numpy(Y)

    def gram(self, A, B):
        return A.double() @ B.double().T

    def factor_gram(self, G2, ell, eps):
        # the ell x ell part of Algorithm 1 from the Gram of [Omega | Y]
        G2 = G2.numpy()
        OO, OY, YY = G2[:ell, :ell], G2[:ell, ell:], G2[ell:, ell:]
        v = eps * np.sqrt(np.trace(OO))
        C = np.linalg.cholesky(0.5 * (OY + OY.T) + v * OO)
        H = YY + v * (OY + OY.T) + v * v * OO
        Ci = np.linalg.inv(C)
        lam, V = np.linalg.eigh(Ci @ H @ Ci.T)
        lam, V = lam[::-1], V[:, ::-1]
        W = Ci.T @ V / np.sqrt(lam)
        return torch.from_numpy(W.copy()), torch.from_numpy(np.maximum(0.0, lam - v)), float(v)

    def tall(self, Y, Om, v, W):
        return W.T @ (Y + v * Om)

    def precond(self, U, S_hat, K, mu=0.0, sqrt_shift=True):
        from oracle.nystrom import precond_weights
        d = precond_weights(S_hat.numpy(), mu, sqrt_shift)
        sd = np.sqrt(d)
        Minv = np.linalg.inv(np.eye(len(d)) + sd[:, None] * K.numpy() * sd[None, :])
        return dict(U=U, d=d, M=sd[:, None] * Minv * sd[None, :])

    def precond_partial(self, pc, z):
        return (pc["U"] @ z.double().reshape(-1)).reshape(1, -1)

    def precond_finish(self, pc, w, z, inverse):
        c = (pc["M"] @ w.numpy().reshape(-1)) if inverse else pc["d"] * w.numpy().reshape(-1)
        return z.double().reshape(-1) + (-1.0 if inverse else 1.0) * (pc["U"].T @ torch.from_numpy(c))


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_2411_08178_gb300.sharded import sharded_factor, sharded_precond_inverse
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        be = NumpyBackend(N1)
        f = sharded_factor(be, N1 * N1, ELL, SEED, EPS, align=8)
        a, b = f["rows"]
        pc = be.precond(f["U"], f["S_hat"], f["K"], 0.0, False)
        z = torch.from_numpy(np.random.default_rng(9).standard_normal(N1 * N1)[a:b].copy())
        pinv = sharded_precond_inverse(be, pc, z)
        q.put((rank, f["rows"], f["U"].numpy(), f["S_hat"].numpy(), f["K"].numpy(), pinv.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_factor_matches_single_rank_oracle(world):
    import oracle
    from oracle import operators as O
    from oracle.philox import gaussian_matrix
    from workloads import gaussian_kernel
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        rank, rows, U, S, K, pinv = q.get(timeout=180)
        got[rank] = (rows, U, S, K, pinv)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the row slices tile the image; every rank has the same S_hat and K
    from paper_2411_08178_gb300.sharded import split
    assert [tuple(got[r][0]) for r in range(world)] == split(N1 * N1, world, 8)
    U = np.concatenate([got[r][1] for r in range(world)], axis=1)
    for r in range(1, world):
        assert np.array_equal(got[r][2], got[0][2]) and np.array_equal(got[r][3], got[0][3])
    # against Algorithm 1 on the whole problem (QR + SVD route of the oracle)
    opo = O.Operator("blur", N1, N1, kernel=gaussian_kernel(5, 1.2))
    phi = lambda V: opo.normal(V.reshape(-1, N1, N1)).reshape(V.shape[0], -1)
    ref = oracle.nystrom.nystrom(phi, gaussian_matrix(N1 * N1, ELL, SEED), EPS)
    S = got[0][2]
    assert np.max(np.abs(S - ref["S_hat"])) <= 1e-9 * ref["S_hat"][0]
    Z = np.random.default_rng(1).standard_normal((4, N1 * N1))
    A_g = ((Z @ U.T) * S) @ U
    A_r = ((Z @ ref["U"].T) * ref["S_hat"]) @ ref["U"]
    assert np.linalg.norm(A_g - A_r) <= 1e-9 * np.linalg.norm(A_r)
    assert np.allclose(got[0][3], U @ U.T, rtol=0, atol=1e-12)
    # the split P^{-1}: the ranks' rows assemble the oracle's P^{-1} z
    P = oracle.nystrom.Precond(ref["U"], ref["S_hat"], 0.0, False)
    z = np.random.default_rng(9).standard_normal(N1 * N1)
    pinv = np.concatenate([got[r][4] for r in range(world)])
    assert np.linalg.norm(pinv - P.inverse(z)) <= 1e-9 * np.linalg.norm(z)


def test_split_shares():
    from paper_2411_08178_gb300.sharded import split
    assert split(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert split(576, 3, 8) == [(0, 192), (192, 384), (384, 576)]
    assert split(20, 3, 8) == [(0, 8), (8, 16), (16, 20)]
    for n, w, a in [(1000, 7, 8), (262144, 8, 8), (37, 2, 1)]:
        s = split(n, w, a)
        assert s[0][0] == 0 and s[-1][1] == n
        assert all(s[i][1] == s[i + 1][0] for i in range(w - 1))
        assert all((b - a0) % a == 0 for a0, b in s[:-1])
