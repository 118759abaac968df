"""Shared helpers of the GPU parity tests (imported by tests marked gpu only)."""
import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2411_08178_gb300 import api
    return torch, api


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# tolerances: float32 operators and preconditioner applies 1e-5 relative per
# apply; float64 paths are held to 1e-12 (rounding of a few thousand terms)
TOL = {"f32": 1e-5, "f64": 1e-12}
