"""GPU parity of the operators (blur, blur + decimation, Joseph ray transform, Haar)
against the float64 oracle, element by element, through the C ABI."""
import math

import numpy as np
import pytest

from oracle import operators as O
from workloads import gaussian_kernel, gaussian_probe_like, random_kernel
from tests.gpu_util import TOL, close, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, api = require_gpu()
    return torch, api, api.Context(0)


DT = {"f32": "float32", "f64": "float64"}


def _t(torch, a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to(getattr(torch, DT[dt])).cuda()


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("shape,kern", [((64, 64), "gauss9"), ((70, 45), "gauss25"), ((33, 97), "rand5"),
                                        ((16, 16), "gauss25"), ((128, 80), "rand7x3")])
def test_blur_apply_adjoint_normal(env, dt, shape, kern):
    torch, api, ctx = env
    n1, n2 = shape
    h = {"gauss9": gaussian_kernel(9, 1.5), "gauss25": gaussian_kernel(25, 4.0), "rand5": random_kernel(5, 1),
         "rand7x3": random_kernel(7, 2)[:, 2:5] / random_kernel(7, 2)[:, 2:5].sum()}[kern]
    op = api.Operator(ctx, "blur", n1, n2, dtype=getattr(torch, DT[dt]), kernel=h)
    x = gaussian_probe_like((3, n1, n2), seed=5)
    xg = _t(torch, x, dt)
    tol = TOL[dt] * (3 if dt == "f32" else 1)
    close(api.op_apply(op, xg).cpu(), O.blur_apply(x, h), tol)
    close(api.op_adjoint(op, xg).cpu(), O.blur_adjoint(x, h), tol)
    close(api.op_normal(op, xg).cpu(), O.blur_adjoint(O.blur_apply(x, h), h), tol)


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_decim_apply_adjoint_normal(env, dt):
    torch, api, ctx = env
    n, d = 64, 4
    h = gaussian_kernel(7, 2.0)
    op = api.Operator(ctx, "blur_decim", n, n, dtype=getattr(torch, DT[dt]), kernel=h, decim=d)
    x = gaussian_probe_like((2, n, n), seed=6)
    yv = gaussian_probe_like((2, n // d, n // d), seed=7)
    close(api.op_apply(op, _t(torch, x, dt)).cpu(), O.decim_apply(x, h, d), TOL[dt])
    close(api.op_adjoint(op, _t(torch, yv, dt)).cpu(), O.decim_adjoint(yv, h, d), TOL[dt])
    close(api.op_normal(op, _t(torch, x, dt)).cpu(), O.decim_adjoint(O.decim_apply(x, h, d), h, d), TOL[dt])


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("geom", [(48, 48, 30, 70), (40, 56, 17, 81), (24, 24, 4, 40)])
def test_radon_apply_adjoint(env, dt, geom):
    torch, api, ctx = env
    n1, n2, na, nb = geom
    op = api.Operator(ctx, "radon", n1, n2, dtype=getattr(torch, DT[dt]), n_angles=na, n_bins=nb)
    x = gaussian_probe_like((2, n1, n2), seed=8)
    s = gaussian_probe_like((2, na, nb), seed=9)
    tol = 1e-5 if dt == "f32" else 1e-12
    close(api.op_apply(op, _t(torch, x, dt)).cpu(), O.radon_apply(x, na, nb), tol)
    close(api.op_adjoint(op, _t(torch, s, dt)).cpu(), O.radon_adjoint(s, n1, n2), tol)
    # exact transposition on the device: <A x, s> = <x, A^T s>
    Ax = api.op_apply(op, _t(torch, x, dt)).double()
    Ats = api.op_adjoint(op, _t(torch, s, dt)).double()
    lhs = float((Ax.cpu().numpy() * s).sum())
    rhs = float((x * Ats.cpu().numpy()).sum())
    assert abs(lhs - rhs) <= (1e-5 if dt == "f32" else 1e-12) * np.linalg.norm(Ax.cpu().numpy()) * np.linalg.norm(s)


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_radon_batch_groups(env, dt):
    # five images: one group of four (the IB = 4 kernels) and a remainder
    torch, api, ctx = env
    n1, n2, na, nb = 40, 56, 17, 81
    op = api.Operator(ctx, "radon", n1, n2, dtype=getattr(torch, DT[dt]), n_angles=na, n_bins=nb)
    x = gaussian_probe_like((5, n1, n2), seed=18)
    s = gaussian_probe_like((5, na, nb), seed=19)
    tol = 1e-5 if dt == "f32" else 1e-12
    close(api.op_apply(op, _t(torch, x, dt)).cpu(), O.radon_apply(x, na, nb), tol)
    close(api.op_adjoint(op, _t(torch, s, dt)).cpu(), O.radon_adjoint(s, n1, n2), tol)
    close(api.op_normal(op, _t(torch, x, dt)).cpu(), O.radon_adjoint(O.radon_apply(x, na, nb), n1, n2), tol)


def test_radon_full_size_properties(env):
    # the 512 x 512, 720 x 736 geometry: at theta = 0 each bin is a column sum
    # (u = m - 112 is an integer, so Joseph's weights are exactly 0 and 1), and
    # <A x, s> = <x, A^T s> in float64 on the host
    torch, api, ctx = env
    n, na, nb = 512, 720, 736
    op = api.Operator(ctx, "radon", n, n, dtype=torch.float32, n_angles=na, n_bins=nb)
    x = gaussian_probe_like((3, n, n), seed=20).astype(np.float32)
    s = gaussian_probe_like((3, na, nb), seed=21).astype(np.float32)
    Ax = api.op_apply(op, torch.from_numpy(x).cuda()).double().cpu().numpy()
    Ats = api.op_adjoint(op, torch.from_numpy(s).cuda()).double().cpu().numpy()
    cols = x.astype(np.float64).sum(axis=1)                  # (3, n)
    assert np.abs(Ax[:, 0, 112:112 + n] - cols).max() <= 1e-4 * np.abs(cols).max()
    assert np.abs(Ax[:, 0, :112]).max() == 0.0 and np.abs(Ax[:, 0, 112 + n:]).max() == 0.0
    lhs = float((Ax * s).sum())
    rhs = float((x * Ats).sum())
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(Ax) * np.linalg.norm(s)


def test_radon_full_size_matches_oracle(env):
    # the 512 x 512, 720-angle, 736-bin projector of the CT workload against
    # the oracle's Joseph projector and its transpose, every angle and bin, in
    # the launch configurations the sketch (a batch of images) and the solver
    # (one image) use
    torch, api, ctx = env
    n, na, nb = 512, 720, 736
    op = api.Operator(ctx, "radon", n, n, dtype=torch.float32, n_angles=na, n_bins=nb)
    x = gaussian_probe_like((n, n), seed=22)
    s = gaussian_probe_like((na, nb), seed=23)
    ref_fwd = O.radon_apply(x, na, nb)
    ref_adj = O.radon_adjoint(s, n, n)
    close(api.op_apply(op, _t(torch, x, "f32")).cpu(), ref_fwd, 1e-5)
    close(api.op_adjoint(op, _t(torch, s, "f32")).cpu(), ref_adj, 1e-5)
    # the same image among five (the 4-images-per-CTA kernels and a remainder)
    xb = np.stack([x, -x, 0.5 * x, x, 2.0 * x])
    sb = np.stack([s, s, -s, 0.25 * s, s])
    fb = api.op_apply(op, _t(torch, xb, "f32")).cpu().numpy()
    ab = api.op_adjoint(op, _t(torch, sb, "f32")).cpu().numpy()
    for b, (cx, cs) in enumerate(zip((1.0, -1.0, 0.5, 1.0, 2.0), (1.0, 1.0, -1.0, 0.25, 1.0))):
        close(fb[b], cx * ref_fwd, 1e-5)
        close(ab[b], cs * ref_adj, 1e-5)


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_haar_forward_inverse(env, dt):
    torch, api, ctx = env
    n = 64
    op = api.Operator(ctx, "blur", n, n, dtype=getattr(torch, DT[dt]), kernel=gaussian_kernel(9, 1.5),
                      haar_levels=3)
    x = gaussian_probe_like((3, n, n), seed=10)
    w = api.op_haar(op, _t(torch, x, dt))
    close(w.cpu(), O.haar_forward(x, 3), TOL[dt])
    close(api.op_haar(op, _t(torch, x, dt), inverse=True).cpu(), O.haar_adjoint(x, 3), TOL[dt])
    close(api.op_haar(op, w, inverse=True).cpu(), x, TOL[dt])


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("shape,levels", [((64, 64), 3), ((32, 48), 2), ((16, 8), 3), ((128, 64), 4)])
def test_daubechies4_forward_inverse(env, dt, shape, levels):
    # the periodic four-tap transform against the oracle's filter bank, down
    # to 2 x 1 coarsest blocks (periodised filters), and W^T W = I
    torch, api, ctx = env
    n1, n2 = shape
    op = api.Operator(ctx, "blur", n1, n2, dtype=getattr(torch, DT[dt]), kernel=gaussian_kernel(3, 1.0),
                      haar_levels=levels, wavelet="db4")
    x = gaussian_probe_like((2, n1, n2), seed=12)
    w = api.op_haar(op, _t(torch, x, dt))
    close(w.cpu(), O.wavelet_forward(x, levels, "db4"), TOL[dt])
    close(api.op_haar(op, _t(torch, x, dt), inverse=True).cpu(), O.wavelet_adjoint(x, levels, "db4"), TOL[dt])
    close(api.op_haar(op, w, inverse=True).cpu(), x, TOL[dt])


def test_unknown_wavelet_is_refused(env):
    torch, api, ctx = env
    from paper_2411_08178_gb300 import _abi as A
    d = A.nys_op_desc()
    d.kind, d.dtype, d.n1, d.n2, d.haar_levels, d.wavelet = A.NYS_OP_RADON, A.NYS_F32, 16, 16, 2, 7
    d.n_angles, d.n_bins, d.angle_span = 8, 24, 3.141592653589793
    import ctypes as C
    h = C.c_void_p()
    assert api._lib().nys_op_create(ctx.h, C.byref(d), C.byref(h)) == A.NYS_EINVAL


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("n1,n2,A,B", [(24, 24, 9, 40), (20, 28, 7, 47)])
def test_fanbeam_matches_oracle(env, dt, n1, n2, A, B):
    # the fan-beam pair (point source at R = 30, flat detector at D = 60,
    # unit bins, full circle) against the oracle, and its dot-product test
    torch, api, ctx = env
    R, D, du = 30.0, 60.0, 1.0
    op = api.Operator(ctx, "fanbeam", n1, n2, dtype=getattr(torch, DT[dt]), n_angles=A, n_bins=B, src_dist=R,
                      det_dist=D, det_spacing=du)
    x = gaussian_probe_like((2, n1, n2), seed=21)
    s = gaussian_probe_like((2, A, B), seed=22)
    ya = api.op_apply(op, _t(torch, x, dt))
    close(ya.cpu(), O.fanbeam_apply(x, A, B, R, D, du), TOL[dt])
    xa = api.op_adjoint(op, _t(torch, s, dt))
    close(xa.cpu(), O.fanbeam_adjoint(s, n1, n2, R, D, du), TOL[dt])
    xn = api.op_normal(op, _t(torch, x, dt))
    close(xn.cpu(), O.fanbeam_adjoint(O.fanbeam_apply(x, A, B, R, D, du), n1, n2, R, D, du), TOL[dt])
    lhs = float((ya.double().cpu() * torch.from_numpy(s)).sum())
    rhs = float((torch.from_numpy(x) * xa.double().cpu()).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12 if dt == "f64" else 1e-5)


def test_fanbeam_geometry_is_validated(env):
    torch, api, ctx = env
    from paper_2411_08178_gb300._abi import NYS_EINVAL, NysError
    for kw in (dict(src_dist=10.0, det_dist=40.0), dict(src_dist=30.0, det_dist=20.0), dict(src_dist=30.0, det_dist=60.0,
                                                                                            det_spacing=0.0)):
        with pytest.raises(NysError) as e:
            api.Operator(ctx, "fanbeam", 24, 24, n_angles=8, n_bins=30, **kw)
        assert e.value.code == NYS_EINVAL


def test_blur_full_size_sampled(env):
    # the 512 x 512, 25 x 25 sigma = 4 operator at full size, checked on
    # sampled pixels that the oracle computes one by one
    torch, api, ctx = env
    n = 512
    h = gaussian_kernel(25, 4.0)
    op = api.Operator(ctx, "blur", n, n, dtype=torch.float32, kernel=h)
    x = gaussian_probe_like((2, n, n), seed=11)
    y = api.op_normal(op, _t(torch, x, "f32")).cpu().numpy()
    rng = np.random.default_rng(0)
    pts = rng.integers(0, n, size=(40, 2))
    pts = np.vstack([pts, [[0, 0], [511, 511], [0, 511], [255, 3]]])
    # H^T H x at (i, j) = sum_{a,b,a',b'} h[a,b] h[a',b'] x[i - a + a', j - b + b'] (periodic)
    kh = h.shape[0]
    c = (kh - 1) // 2
    for b in range(2):
        for (i, j) in pts:
            # Hx on the neighbourhood rows/cols needed, then H^T at (i, j)
            acc = 0.0
            for a in range(kh):
                for bb in range(kh):
                    ii, jj = (i - a + c) % n, (j - bb + c) % n
                    rows = (ii + np.arange(kh) - c) % n
                    cols = (jj + np.arange(kh) - c) % n
                    acc += h[a, bb] * float((h * x[b][np.ix_(rows, cols)]).sum())
            assert abs(y[b, i, j] - acc) <= 1e-5 * max(1.0, abs(acc)), (b, i, j)
