"""Algorithm 1 and the preconditioner spread over torch.distributed ranks.

The probe columns of the sketch are independent (Sec. III-C), so each rank
draws and sketches its own slice of them; the tall-skinny algebra after it
needs every column of a pixel, so the slices are then exchanged into pixel
slices.  Per call, with `world` ranks:

  1. rank r draws columns J_r of Omega and computes Y = Phi Omega for them
     (nys_sketch_cols): the operator work is split by columns;
  2. one all-to-all turns the column slices into row slices: rank r then holds
     rows I_r (its pixels) of every column of Omega and Y;
  3. each rank forms the Gram of its rows of [Omega | Y]; one all-reduce (sum)
     of the (2 ell)^2 float64 Gram gives the full Gram on every rank;
  4. every rank runs the ell x ell part of Algorithm 1 on it
     (nys_factor_gram: shift, shifted Cholesky, eigen-decomposition): the
     inputs are identical, so are W, S_hat and v;
  5. each rank forms its rows of U = (Y + v Omega) W (nys_tall_gemm) and the
     Gram of its rows of U; one all-reduce gives K = U^T U;
  6. the preconditioner P = I + U diag(d) U^T is set up from K on every rank
     (nys_precond_import_gram); P^{-1} z for a pixel-sharded z is
     precond_partial, an all-reduce of the ell_active sums, precond_finish.

The collectives are torch.distributed calls on the backend's tensors (NCCL
for device tensors).  The local steps go through a backend object, so that
the exchange pattern is the same code whatever computes the local steps;
`DeviceBackend` is the library on the GPU.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def split(n: int, world: int, align: int = 1) -> list[tuple[int, int]]:
    """[start, stop) of each rank's share of n items, shares a multiple of
    `align` except the last, as equal as that allows."""
    units = -(-n // align)
    base, extra = divmod(units, world)
    out, start = [], 0
    for r in range(world):
        stop = min(n, start + (base + (1 if r < extra else 0)) * align)
        out.append((start, stop))
        start = stop
    return out


def _world(group):
    if group is None and not (dist.is_available() and dist.is_initialized()):
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def _all_reduce(t: torch.Tensor, group, world: int) -> torch.Tensor:
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def columns_to_rows(Xc: torch.Tensor, cols, rows, rank: int, group, world: int) -> torch.Tensor:
    """Xc: (ell_r, N) this rank's columns -> (ell, N_r) every column's rows of
    this rank (one all-to-all)."""
    if world == 1:
        return Xc.contiguous()
    send = torch.cat([Xc[:, a:b].reshape(-1) for (a, b) in rows])
    in_sizes = [Xc.shape[0] * (b - a) for (a, b) in rows]
    r0, r1 = rows[rank]
    out_sizes = [(c1 - c0) * (r1 - r0) for (c0, c1) in cols]
    recv = torch.empty(sum(out_sizes), dtype=Xc.dtype, device=Xc.device)
    dist.all_to_all_single(recv, send, out_sizes, in_sizes, group=group)
    return recv.reshape(cols[-1][1], r1 - r0)


def sharded_factor(backend, N: int, ell: int, seed: int, eps: float, group=None, align: int = 8) -> dict:
    """Steps 1-5 above on this rank.  Returns dict(U = this rank's rows of U
    (ell, N_r), S_hat, K, v, rows = (start, stop), Omega, Y = this rank's rows
    of Omega and Y)."""
    rank, world = _world(group)
    cols = split(ell, world)
    rows = split(N, world, align)
    j0, j1 = cols[rank]
    if j1 <= j0 or rows[rank][1] <= rows[rank][0]:
        raise ValueError("sharded_factor: every rank needs at least one column and one row")
    Om_c, Y_c = backend.sketch_cols(ell, j0, j1, seed)
    Om = columns_to_rows(Om_c.reshape(j1 - j0, N), cols, rows, rank, group, world)
    Y = columns_to_rows(Y_c.reshape(j1 - j0, N), cols, rows, rank, group, world)
    G2 = torch.zeros((2 * ell, 2 * ell), dtype=torch.float64, device=Om.device)
    G2[:ell, :ell] = backend.gram(Om, Om)
    G2[:ell, ell:] = backend.gram(Om, Y)
    G2[ell:, ell:] = backend.gram(Y, Y)
    _all_reduce(G2, group, world)
    W, S_hat, v = backend.factor_gram(G2, ell, eps)
    U = backend.tall(Y, Om, v, W)
    K = _all_reduce(backend.gram(U, U), group, world)
    return dict(U=U, S_hat=S_hat, K=K, v=v, rows=rows[rank], Omega=Om, Y=Y)


def sharded_precond_inverse(backend, pc, z: torch.Tensor, group=None, inverse: bool = True) -> torch.Tensor:
    """This rank's rows of P^{-1} z (P z with inverse=False) for this rank's
    rows z of a pixel-sharded vector (step 6)."""
    rank, world = _world(group)
    w = _all_reduce(backend.precond_partial(pc, z), group, world)
    return backend.precond_finish(pc, w, z, inverse)


class DeviceBackend:
    """The local steps on the GPU, through the library (Context, Operator)."""

    def __init__(self, ctx, op, store_dtype=torch.bfloat16, u_dtype=None):
        from . import api
        self.api, self.ctx, self.op = api, ctx, op
        self.sd = store_dtype
        self.ud = u_dtype or store_dtype

    def sketch_cols(self, ell, j0, j1, seed):
        return self.api.nys_sketch_cols(self.ctx, self.op, ell, j0, j1, seed, store_dtype=self.sd)

    def gram(self, A, B):
        return self.api.nys_gram(self.ctx, A.contiguous(), B.contiguous())

    def factor_gram(self, G2, ell, eps):
        W, S, v, _ = self.api.nys_factor_gram(self.ctx, G2, ell, eps, eig_f64=self.sd == torch.float64)
        return W, S, v

    def tall(self, Y, Om, v, W):
        return self.api.nys_tall_gemm(self.ctx, Y.contiguous(), Om.contiguous(), v, W, out_dtype=self.ud)

    def precond(self, U, S_hat, K, mu=0.0, sqrt_shift=True):
        pc = self.api.Precond(self.ctx, U.shape[1], U.shape[0], self.ud)
        return pc.import_gram(U, S_hat, K, mu, sqrt_shift)

    def precond_partial(self, pc, z):
        return self.api.precond_partial(self.ctx, pc, z)

    def precond_finish(self, pc, w, z, inverse):
        return self.api.precond_finish(self.ctx, pc, w, z, inverse)
