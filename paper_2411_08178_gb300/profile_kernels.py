"""Per-call timings of the library's hot entry points, and a small target for ncu.

  python -m paper_2411_08178_gb300.profile_kernels [--case all|precond|normal|sketch|prox|prox_mixed|irm|iter|unroll|batch]
        [--n 512] [--ell 200] [--reps 20] [--l2] [--dual-stop off|on]

Each case builds the 512 x 512 deblurring operator (25 x 25 Gaussian, sigma 4)
and times one library call with CUDA events on the calling stream (warm-up
first, mean over --reps), then prints one JSON line per case with the time
and the algorithmic bytes or flops of the call.  With few repetitions it is
also the workload for `ncu -k regex:<kernel> -c <n>` captures.  The exact
early stop of the dual iterations is off unless --dual-stop on: the prox
cases then time every dual step (their cost per step), whatever the input.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="all")
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--ell", type=int, default=200)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--u-dtype", choices=["bf16", "f32"], default="bf16")
    ap.add_argument("--l2", action="store_true", help="keep U resident in L2 (nys_l2_persist)")
    ap.add_argument("--dual-stop", choices=["off", "on"], default="off",
                    help="the exact early stop of the dual iterations (off: every dual step runs)")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-inner", type=int, default=20)
    ap.add_argument("--irm-eps", type=float, default=1e-8, help="IRM smoothing |r|_eps = sqrt(r^2 + eps)")
    ap.add_argument("--irm-lambda", type=float, default=2e-3)
    ap.add_argument("--op", choices=["blur", "radon", "fanbeam"], default="blur",
                    help="blur: 25 x 25 Gaussian sigma 4; radon: 720 angles x 736 bins; fanbeam: 720 angles over "
                         "360 deg x 1024 bins, source at 1000, detector at 2000 pixels")
    args = ap.parse_args()
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2411_08178_gb300 import api
    import workloads as WL

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = api.Context(0, stream)
    ctx.set_dual_stop(args.dual_stop == "on")
    n, ell = args.n, args.ell
    N = n * n
    if args.op == "blur":
        op = api.Operator(ctx, "blur", n, n, dtype=torch.float32, kernel=WL.gaussian_kernel(25, 4.0))
    elif args.op == "radon":
        op = api.Operator(ctx, "radon", n, n, dtype=torch.float32, n_angles=720, n_bins=736)
    else:
        op = api.Operator(ctx, "fanbeam", n, n, dtype=torch.float32, n_angles=720, n_bins=1024, src_dist=1000.0,
                          det_dist=2000.0)
    sd = torch.bfloat16 if args.u_dtype == "bf16" else torch.float32
    ub = 2 if sd == torch.bfloat16 else 4

    def timed(fn, reps=args.reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    out = []
    Om, Y = api.nys_sketch(ctx, op, ell, 13, store_dtype=sd)
    pc = api.nys_factor(ctx, Om, Y, 2.0 ** -23, u_dtype=sd)
    if args.l2:
        ctx.l2_persist(pc.U, 1.0)
    cases = args.case.split(",") if args.case != "all" else ["precond", "normal", "sketch", "prox", "iter"]
    if "precond" in cases:
        z = torch.randn(N, device=dev)
        o = torch.empty_like(z)
        ms = timed(lambda: api.precond_apply(ctx, pc, z, True, o))
        nbytes = 2 * N * pc.ell_active * ub + 3 * N * 4
        out.append(dict(case="precond_apply(inverse)", ms=ms, bytes=nbytes, GBs=nbytes / ms / 1e6,
                        active_columns=pc.ell_active))
    if "normal" in cases:
        x1 = torch.randn(1, n, n, device=dev)
        y1 = torch.empty_like(x1)
        ms = timed(lambda: api.op_normal(op, x1, y1))
        out.append(dict(case=f"op_normal x1 ({args.op})", ms=ms, bytes=2 * N * 4))
    if "sketch" in cases:
        ms = timed(lambda: api.nys_sketch(ctx, op, ell, 13, store_dtype=sd, out=(Om, Y)), reps=max(2, args.reps // 4))
        out.append(dict(case=f"nys_sketch ell={ell} ({args.op})", ms=ms, bytes=2 * N * ell * ub))
        ms = timed(lambda: api.nys_factor(ctx, Om, Y, 2.0 ** -23, pc=pc), reps=max(2, args.reps // 4))
        out.append(dict(case=f"nys_factor ell={ell}", ms=ms, bytes=4 * N * ell * ub, flops=4 * 2 * N * ell * ell))
    if "prox" in cases:
        s = torch.rand(n, n, device=dev)
        Q = torch.zeros(2, n, n, device=dev)
        ms = timed(lambda: api.prox_tv(ctx, None, 5e-4, 20, s, Q=Q), reps=max(2, args.reps // 2))
        out.append(dict(case="prox_tv P=I n_inner=20", ms=ms))
        ms = timed(lambda: api.prox_tv(ctx, pc, 5e-4, 20, s, Q=Q), reps=max(2, args.reps // 2))
        out.append(dict(case="prox_tv P=RNP n_inner=20", ms=ms))
    if "prox_mixed" in cases:
        # every mixed-norm regulariser, P = I and P = RNP, 20 dual steps; the
        # algorithmic bytes of one dual step as the launches stream them:
        # anisotropic TV fuses the update (x, old and new (R, Q), s, x / g),
        # the others read R for L^T, then x, R, Q for the update
        s = torch.rand(n, n, device=dev)
        for reg in ("tv", "isotv", "hs", "hs2", "hsinf"):
            G = 2 if reg in ("tv", "isotv") else 3
            Q = torch.zeros(G, n, n, device=dev)
            for name, p_ in (("P=I", None), ("P=RNP", pc)):
                ms = timed(lambda: api.prox_mixed(ctx, p_, reg, 5e-4, 20, s, Q=Q), reps=max(2, args.reps // 2))
                if p_ is None:
                    words = 4 * G + 3 if reg == "tv" else 5 * G + 3
                    per_step = words * N * 4
                else:
                    words = 4 * G + 5 if reg == "tv" else 5 * G + 5
                    per_step = words * N * 4 + 2 * pc.ell_active * N * ub
                out.append(dict(case=f"prox_mixed {reg} {name} n_inner=20", ms=ms, bytes=21 * per_step,
                                GBs=21 * per_step / ms / 1e6, active_columns=pc.ell_active if p_ is not None else 0))
    if "irm" in cases:
        # Algorithm 2 on the impulsive-noise deblurring setting of the
        # experiments: 512 x 512, 9 x 9 Gaussian (sigma 1.6) or uniform blur,
        # 5% + 5% salt and pepper, q = 1, p in {1, 0.5}, PCG tolerance 1e-4,
        # 5 outer iterations, plain CG against ell = 100 (bf16 sketch); wall
        # time of the 5 outer iterations (sketches and factors included)
        import numpy as np
        rng = np.random.default_rng(51)
        xt = torch.from_numpy(WL.phantom(n, 30, 51, "ellipse")).float().to(dev)
        for blur_name, hk in (("gauss9 s1.6", WL.gaussian_kernel(9, 1.6)), ("uniform9", np.full((9, 9), 1.0 / 81))):
            opi = api.Operator(ctx, "blur", n, n, dtype=torch.float32, kernel=hk)
            yv = api.op_apply(opi, xt[None])[0].double().cpu().numpy()
            msk = rng.uniform(size=(n, n))
            yv = np.where(msk < 0.05, 1.0, np.where(msk > 0.95, 0.0, yv))
            yt = torch.from_numpy(yv).float().to(dev)
            for pp in (1.0, 0.5):
                res = {}
                for ell_i in (0, 100):
                    irm = api.IRM(ctx, opi, yt, pp, 1.0, args.irm_lambda, args.irm_eps, ell=ell_i, store_dtype=sd,
                                  seed=7, cg_tol=1e-4, cg_max=20000)
                    irm.step()                      # warm-up (sizes scratch, loads kernels)
                    irm.reset()
                    torch.cuda.synchronize()
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    its = [irm.step()["cg_iters"] for _ in range(5)]
                    b.record(stream)
                    torch.cuda.synchronize()
                    res[ell_i] = (a.elapsed_time(b), its)
                    irm.close()
                t0, t1 = res[0][0], res[100][0]
                out.append(dict(case=f"irm {blur_name} p={pp} q=1 lambda={args.irm_lambda} eps={args.irm_eps} "
                                     f"5 outer iterations", ms_plain=t0, ms_rnp=t1, cg_plain=res[0][1],
                                cg_rnp=res[100][1], saved_time=(t0 - t1) / t0,
                                saved_cg=1.0 - sum(res[100][1]) / sum(res[0][1])))
            opi.close()
    if "read_ceiling" in cases:
        # DRAM bandwidth of a read-only stream against a read + write copy,
        # over U's size (ell bf16 images): torch's sum and clone, CUDA events,
        # a 256 MB write between repetitions so that every byte comes from DRAM
        big = torch.zeros(ell * N, dtype=torch.bfloat16, device=dev)
        acc = torch.empty(ell * N // 4096, dtype=torch.float32, device=dev)
        dst = torch.empty_like(big)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

        def flushed(fn, reps=args.reps):
            ts = []
            for r in range(reps + 3):
                flush.fill_(float(r))
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                torch.cuda.synchronize()
                if r >= 3:
                    ts.append(a.elapsed_time(b))
            return sum(ts) / len(ts)
        nb = ell * N * 2
        ms = flushed(lambda: torch.sum(big.view(-1, 4096), dim=1, dtype=torch.float32, out=acc))
        out.append(dict(case=f"read-only stream (row sums of {nb / 1e6:.0f} MB bf16, rows of 4096)", ms=ms, bytes=nb,
                        GBs=nb / ms / 1e6))
        # the library matrix-vector product over the same bytes: U^T z with U
        # as an ell x N bf16 matrix (what the U^T g pass computes)
        zv = torch.zeros(N, dtype=torch.bfloat16, device=dev)
        yv = torch.empty(ell, dtype=torch.bfloat16, device=dev)
        ms = flushed(lambda: torch.mv(big.view(ell, N), zv, out=yv))
        out.append(dict(case=f"read-only stream (torch.mv, {ell} x {N} bf16)", ms=ms, bytes=nb, GBs=nb / ms / 1e6))
        ms = flushed(lambda: dst.copy_(big))
        out.append(dict(case=f"copy (read + write {nb / 1e6:.0f} MB each)", ms=ms, bytes=2 * nb, GBs=2 * nb / ms / 1e6))
        del big, dst, flush
    if "iter" in cases:
        y = torch.rand(op.meas_shape, device=dev)
        for name, p in (("plain", None), ("precond", pc)):
            sol = api.Solver(ctx, op, y, "tv", 5e-4, pc=p, n_inner=20)
            ms = timed(lambda: sol.step(1), reps=args.reps)
            out.append(dict(case=f"pgd_step TV {name}", ms=ms))
            sol.close()
    if "unroll" in cases:
        # 50 unrolled preconditioned iterations (n_inner 20), checkpoint every 10:
        # forward alone and forward + reverse pass (d/d lambda, d/d 25x25 kernel)
        y = torch.rand(op.meas_shape, device=dev)
        un = api.Unroll(ctx, op, 5e-4, 0.9, 50, n_inner=20, ckpt_every=10, pc=pc)
        xb = torch.randn(n, n, device=dev)
        ms_f = timed(lambda: un.forward(y), reps=2)
        ms_fb = timed(lambda: (un.forward(y), un.backward(xb)), reps=2)
        out.append(dict(case="unroll K=50 n_inner=20 ckpt=10 forward", ms=ms_f))
        out.append(dict(case="unroll K=50 n_inner=20 ckpt=10 forward+backward", ms=ms_fb))
        un.close()
    if "batch" in cases:
        # the batched, differentiated workload: 64 instances (128^2 .. 512^2,
        # blur / CT, ell in {64, 128, 256}), 50 unrolled iterations, checkpoint
        # every 10, one graph launch forward and one backward
        import time
        from paper_2411_08178_gb300.batched import BatchedUnroll
        specs = []
        for inst in WL.batch_instances(args.batch_count):
            sp = dict(inst)
            ctx_i = api.Context(0)
            if inst["op"] == "blur":
                sp["kernel"] = WL.gaussian_kernel(inst["k"], inst["sigma"])
                opi = api.Operator(ctx_i, "blur", inst["n"], inst["n"], dtype=torch.float32, kernel=sp["kernel"])
            else:
                opi = api.Operator(ctx_i, "radon", inst["n"], inst["n"], dtype=torch.float32,
                                   n_angles=inst["n_angles"], n_bins=inst["n_bins"])
            sp["x_true"], sp["y"] = WL.batch_instance_data(
                inst, lambda xt: api.op_apply(opi, torch.from_numpy(xt).float().to(dev)[None]).cpu().numpy()[0])
            opi.close()
            specs.append(sp)
        t0 = time.time()
        B = BatchedUnroll(specs, K=50, n_inner=args.batch_inner, ckpt_every=10)
        setup_s = time.time() - t0
        bs = B.stream

        def timed_on(fn, reps=3):
            fn()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(bs)
            for _ in range(reps):
                fn()
            b.record(bs)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        ms_f = timed_on(B.forward)
        ms_b = timed_on(B.backward)
        pix = sum(sp["n"] ** 2 for sp in specs)
        out.append(dict(case=f"batch {len(specs)} instances K=50 n_inner={args.batch_inner} forward (one graph)",
                        ms=ms_f, pixels=pix, setup_s=round(setup_s, 1)))
        out.append(dict(case=f"batch {len(specs)} instances backward (one graph)", ms=ms_b,
                        tuned=[it["tuned"] for it in B.items]))
    for o in out:
        print(json.dumps(o))


if __name__ == "__main__":
    main()
