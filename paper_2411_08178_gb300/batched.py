"""Set-up of a batch of differentiated unrolled solves (mixed sizes, operators
and sketch sizes) replayed as one CUDA graph.  Every step is a libnys call:
per instance its own Context and stream, the operator (tuned by the project
autotuner), the sketch and Algorithm 1 factor, the power-iteration step size,
and an Unroll handle; then one Batch over all of them."""
from __future__ import annotations

import numpy as np
import torch

from . import api

EPS32 = 2.0 ** -23


class BatchedUnroll:
    """specs: dicts with op ("blur" with kernel, or "radon" with n_angles,
    n_bins), n, ell, lam, seed_omega, and the data y (numpy, measurement
    shape).  K unrolled iterations of n_inner dual steps, checkpoint every
    ckpt_every; float32 iterates, bf16 sketch and U."""

    def __init__(self, specs: list, K: int = 50, n_inner: int = 20, ckpt_every: int = 10, device: int = 0,
                 autotune: bool = True):
        dev = torch.device("cuda", device)
        # the batch stream comes from the high-priority pool, the item streams
        # from the default one (a pool of 32, so items may share a stream and
        # then run one after the other; never the batch stream)
        self.main = api.Context(device, torch.cuda.Stream(dev, priority=-1))
        self.items = []
        for sp in specs:
            stream = torch.cuda.Stream(dev)
            ctx = api.Context(device, stream)
            n = sp["n"]
            if sp["op"] == "blur":
                op = api.Operator(ctx, "blur", n, n, dtype=torch.float32, kernel=sp["kernel"])
            else:
                op = api.Operator(ctx, "radon", n, n, dtype=torch.float32, n_angles=sp["n_angles"],
                                  n_bins=sp["n_bins"])
            tuned = op.autotune(batch=4) if autotune else None
            with torch.cuda.stream(stream):
                Om, Y = api.nys_sketch(ctx, op, sp["ell"], sp["seed_omega"], store_dtype=torch.bfloat16)
                pc = api.Precond(ctx, n * n, sp["ell"], torch.bfloat16)
                api.nys_factor(ctx, Om, Y, EPS32, pc=pc)
                y = torch.from_numpy(np.ascontiguousarray(sp["y"], dtype=np.float32)).to(dev)
                sol = api.Solver(ctx, op, y, "tv", sp["lam"], pc=pc, n_inner=n_inner)
                alpha = sol.alpha
                sol.close()
                un = api.Unroll(ctx, op, sp["lam"], alpha, K, n_inner=n_inner, ckpt_every=ckpt_every, pc=pc)
                x = torch.zeros((n, n), dtype=torch.float32, device=dev)
                xbar = torch.zeros_like(x)
            ctx.sync()
            del Om, Y
            self.items.append(dict(ctx=ctx, stream=stream, op=op, pc=pc, unroll=un, y=y, x=x, xbar=xbar,
                                   alpha=alpha, tuned=tuned, spec=sp))
        self.batch = api.Batch(self.main, [it["unroll"] for it in self.items], [it["y"] for it in self.items],
                               [it["x"] for it in self.items], [it["xbar"] for it in self.items])

    @property
    def stream(self):
        return self.main.stream

    def forward(self):
        self.batch.forward()

    def backward(self):
        self.batch.backward()

    def grads(self):
        return self.batch.grads
