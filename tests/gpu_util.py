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


def _np(a):
    if hasattr(a, "detach"):
        a = a.detach().cpu().double().numpy()
    return np.asarray(a, dtype=np.float64)


def rel(a, b):
    """Norm-wise relative error ||a - b|| / ||b||."""
    a, b = _np(a), _np(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def maxrel(a, b):
    """Element-wise error scaled by the reference's largest entry:
    max |a - b| / max |b|.  A wrong boundary row or wrap-around column moves
    the norm-wise error of a large image by only about 1/sqrt(N); this does not
    average it away."""
    a, b = _np(a), _np(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def close(a, b, tol, el_tol=None):
    """Both the norm-wise and the element-wise error within tolerance."""
    r, m = rel(a, b), maxrel(a, b)
    el = tol if el_tol is None else el_tol
    assert r < tol and m < el, f"norm-wise {r:.3e} (tol {tol:.1e}), element-wise {m:.3e} (tol {el:.1e})"


# tolerances: float32 operators and preconditioner applies 1e-5 relative per
# apply; float64 paths are held to 1e-12 (rounding of a few thousand terms)
TOL = {"f32": 1e-5, "f64": 1e-12}
