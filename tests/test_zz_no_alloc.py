"""precond_apply_noalloc: the allocation-free variant of precond_apply.

Some callers cannot let the library call cudaMalloc -- for example while their
own stream is being captured into a CUDA graph, or under a fixed device memory
budget.  precond_apply_noalloc gives them P and P^{-1} with its scratch in one
fixed device array compiled into the library.  This test calls it through the
C ABI and checks it against precond_apply, twice in a row (the array keeps
the previous call's contents), and checks that a problem too large for the
array is refused with NYS_EINVAL.  It lives in its own file, collected last.
"""
import ctypes as C

import numpy as np
import pytest

from tests.gpu_util import TOL, rel, require_gpu

pytestmark = pytest.mark.gpu


def _call(lib, ctx, pc, inverse, dtype, z, out):
    return lib.precond_apply_noalloc(ctx.h, C.byref(pc.s), int(inverse), dtype, z.data_ptr(), out.data_ptr(),
                                     z.numel() // pc.s.N)


@pytest.mark.parametrize("dt", ["f32", "f64", "bf16u"])
def test_noalloc_matches_precond_apply_twice(dt):
    torch, api = require_gpu()
    from paper_2411_08178_gb300 import _abi
    from workloads import gaussian_kernel, gaussian_probe_like
    lib = _abi.load()
    ctx = api.Context(0)
    n, ell = 96, 24
    tdt = torch.float64 if dt == "f64" else torch.float32
    op = api.Operator(ctx, "blur", n, n, dtype=tdt, kernel=gaussian_kernel(9, 1.5))
    sd = torch.bfloat16 if dt == "bf16u" else tdt
    Om, Y = api.nys_sketch(ctx, op, ell, seed=21, store_dtype=sd)
    pc = api.nys_factor(ctx, Om, Y, 2.0 ** -52 if dt == "f64" else 2.0 ** -23, u_dtype=sd)
    code = _abi.NYS_F64 if dt == "f64" else _abi.NYS_F32
    tol = TOL["f64" if dt == "f64" else "f32"]
    for call in range(2):
        z = torch.from_numpy(gaussian_probe_like((2, n * n), seed=30 + call)).to(tdt).cuda()
        for inverse in (True, False):
            ref = api.precond_apply(ctx, pc, z, inverse=inverse)
            out = torch.full_like(z, float("nan"))
            st = _call(lib, ctx, pc, inverse, code, z, out)
            assert st == _abi.NYS_OK, lib.nys_last_error(ctx.h)
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert rel(out.double().cpu().numpy(), ref.double().cpu().numpy()) <= tol


def test_noalloc_rejects_problems_beyond_the_fixed_array():
    torch, api = require_gpu()
    from paper_2411_08178_gb300 import _abi
    lib = _abi.load()
    ctx = api.Context(0)
    # f64 with every column active (s_i > sqrt(s_K) = sqrt 2):
    # ceil(N/1024) * ell_active + ell_active = 512 * 512 + 512 doubles > 2 MiB
    N, ell = 512 * 1024, 512
    pc = api.Precond(ctx, N, ell, torch.float64)
    pc.U.zero_()
    pc.S_hat.copy_(torch.linspace(4.0, 2.0, ell, dtype=torch.float64))
    assert lib.nys_precond_import(ctx.h, C.byref(pc.s), 0.0, 1) == _abi.NYS_OK
    assert pc.ell_active == ell
    z = torch.ones(N, dtype=torch.float64, device="cuda")
    out = torch.empty_like(z)
    assert _call(lib, ctx, pc, True, _abi.NYS_F64, z, out) == _abi.NYS_EINVAL
    assert b"fixed array" in lib.nys_last_error(ctx.h)
    del pc
    torch.cuda.empty_cache()
