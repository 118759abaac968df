"""Tall-skinny Gram products A^T B (Algorithm 1's Omega^T Omega, Omega^T Y, Y^T Y,
and U^T U) through the C ABI: the tcgen05 tensor-core path and the CUDA-core
path against a float64 matmul of the same bf16 values."""
import numpy as np
import pytest

from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, api = require_gpu()
    return torch, api, api.Context(0)


def _operands(torch, p, q, N, seed, same=False):
    g = torch.Generator(device="cpu").manual_seed(seed)
    A = torch.randn(p, N, generator=g).to(torch.bfloat16)
    B = A.clone() if same else torch.randn(q, N, generator=g).to(torch.bfloat16)
    ref = A.double().numpy() @ B.double().numpy().T
    return A.cuda(), B.cuda(), ref


# (p, q, N): the ell = 200 sketch at 512 x 512, ragged K (N not a multiple of
# the 64-pixel K block), a second M tile that is mostly padding, narrow and
# full-width outputs, a single column, and outputs wider than one 256-column
# tile (two and four column tiles, rows over several 128-row tiles)
CASES = [(200, 200, 262144), (130, 48, 5000), (64, 17, 4096), (128, 256, 8192), (1, 1, 1024), (257, 96, 2048),
         (300, 520, 8192), (400, 400, 20000), (96, 1024, 4096)]


@pytest.mark.parametrize("p,q,N", CASES)
def test_gram_tensor_cores_match_float64(env, p, q, N):
    torch, api, ctx = env
    A, B, ref = _operands(torch, p, q, N, seed=p * 7 + q)
    C = api.nys_gram(ctx, A, B, path=2).cpu().numpy()
    err = np.linalg.norm(C - ref) / np.linalg.norm(ref)
    assert err < 1e-5, err


@pytest.mark.parametrize("p,q,N", CASES[:3])
def test_gram_paths_agree(env, p, q, N):
    torch, api, ctx = env
    A, B, ref = _operands(torch, p, q, N, seed=3)
    Ct = api.nys_gram(ctx, A, B, path=2).cpu().numpy()
    Cc = api.nys_gram(ctx, A, B, path=1).cpu().numpy()
    assert np.linalg.norm(Ct - Cc) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("k,N,out", [(200, 262144, "bf16"), (48, 5000, "f32"), (17, 1024, "f32"), (256, 2048, "bf16"),
                                     (1, 128, "f32"), (400, 16384, "f32"), (600, 4096, "bf16"), (1024, 2048, "f32")])
def test_tall_gemm_tensor_cores_match_float64(env, k, N, out):
    # U = (Y + v Omega) W: the MN-major A operand (columns are images)
    torch, api, ctx = env
    g = torch.Generator(device="cpu").manual_seed(k + N)
    Y = torch.randn(k, N, generator=g).to(torch.bfloat16)
    Om = torch.randn(k, N, generator=g).to(torch.bfloat16)
    W = torch.randn(k, k, generator=g, dtype=torch.float64) / np.sqrt(k)
    v = 0.37
    ref = ((Y.double() + v * Om.double()).T.numpy() @ W.numpy()).T       # (q, N)
    od = torch.bfloat16 if out == "bf16" else torch.float32
    U = api.nys_tall_gemm(ctx, Y.cuda(), Om.cuda(), v, W.cuda(), out_dtype=od, path=2).double().cpu().numpy()
    # bf16 output rounding (2^-9) / W split into bf16 hi + lo (about 2^-17)
    tol = 8e-3 if out == "bf16" else 1e-4
    assert np.linalg.norm(U - ref) / np.linalg.norm(ref) < tol
    Uc = api.nys_tall_gemm(ctx, Y.cuda(), Om.cuda(), v, W.cuda(), out_dtype=od, path=1).double().cpu().numpy()
    assert np.linalg.norm(U - Uc) / np.linalg.norm(ref) < tol


@pytest.mark.parametrize("p,N", [(40, 4096), (300, 8192), (800, 4096)])
def test_gram_symmetric_and_fallback(env, p, N):
    # A^T A of one operand computes only the tiles that reach the diagonal and
    # mirrors them: the full matrix must come back, exactly symmetric
    torch, api, ctx = env
    A, _, ref = _operands(torch, p, p, N, seed=9, same=True)
    C = api.nys_gram(ctx, A, A, path=2).cpu().numpy()
    assert np.array_equal(C, C.T)
    assert np.linalg.norm(C - ref) / np.linalg.norm(ref) < 1e-5
    # N not a multiple of 8 (rows not 16-byte aligned): the tensor-core path declines
    from paper_2411_08178_gb300._abi import NYS_EINVAL, NysError
    A2, B2, ref2 = _operands(torch, 8, 300, 1020, seed=4)
    with pytest.raises(NysError) as e:
        api.nys_gram(ctx, A2, B2, path=2)
    assert e.value.code == NYS_EINVAL
    C2 = api.nys_gram(ctx, A2, B2, path=0).cpu().numpy()
    assert np.linalg.norm(C2 - ref2) / np.linalg.norm(ref2) < 1e-5
