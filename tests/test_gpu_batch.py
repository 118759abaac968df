"""The batched, differentiated workload as one CUDA graph: mixed image sizes,
blur and CT instances, mixed sketch sizes, each instance on its own context
and stream, forward and reverse pass each one graph launch.  The graph's
results must equal, bit for bit, the same instances run one by one through
the C ABI (same kernels, same order within an instance); the project
autotuner's choices must be valid variants."""
import numpy as np
import pytest

import workloads as WL
from oracle import operators as O
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _specs(count=6):
    out = []
    for inst in WL.batch_instances(count, seed=7, sizes=(32, 48), ells=(8, 16), angle_range=(12, 30)):
        sp = dict(inst)
        if inst["op"] == "blur":
            h = WL.gaussian_kernel(inst["k"], inst["sigma"])
            sp["kernel"] = h
            opo = O.Operator("blur", inst["n"], inst["n"], kernel=h)
        else:
            opo = O.Operator("radon", inst["n"], inst["n"], n_angles=inst["n_angles"], n_bins=inst["n_bins"])
        sp["x_true"], sp["y"] = WL.batch_instance_data(inst, opo.apply)
        out.append(sp)
    return out


def test_batch_graph_equals_individual_solves():
    torch, api = require_gpu()
    from paper_2411_08178_gb300.batched import BatchedUnroll
    specs = _specs()
    B = BatchedUnroll(specs, K=4, n_inner=3, ckpt_every=2)
    for it in B.items:
        if it["spec"]["op"] == "radon":
            assert it["tuned"] in (4, 8, 16)
        else:
            assert it["tuned"] in (32, 64)
    B.forward()
    torch.cuda.synchronize()
    xs = [it["x"].clone() for it in B.items]
    with torch.cuda.stream(B.stream):
        for it, x in zip(B.items, xs):
            xt = torch.from_numpy(it["spec"]["x_true"]).float().cuda()
            it["xbar"].copy_(2.0 * (x - xt) / x.numel())
    B.backward()
    torch.cuda.synchronize()
    gb = [g.clone() for g in B.grads()]
    for it, x, g in zip(B.items, xs, gb):
        with torch.cuda.stream(it["stream"]):
            xi = it["unroll"].forward(it["y"])
            dl, dh = it["unroll"].backward(it["xbar"])
        torch.cuda.synchronize()
        assert torch.equal(xi, x)
        assert float(dl) == float(g[0])
        if dh is not None:
            assert torch.equal(dh.reshape(-1), g[1:])
        assert np.isfinite(float(g[0])) and float(g[0]) != 0.0


def test_batch_backward_before_forward_is_refused():
    torch, api = require_gpu()
    from paper_2411_08178_gb300.batched import BatchedUnroll
    from paper_2411_08178_gb300._abi import NYS_EINVAL, NysError
    B = BatchedUnroll(_specs(2), K=2, n_inner=2, ckpt_every=1, autotune=False)
    with pytest.raises(NysError) as e:
        B.backward()
    assert e.value.code == NYS_EINVAL
