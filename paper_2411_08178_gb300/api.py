"""Thin Python binding over libnys.so with the C ABI's names.

Torch is used only for device memory and the current CUDA stream: every
function passes raw pointers and sizes to the library, which does all of the
computation.  Shapes and dtypes are checked here so that errors are caught
before a pointer reaches the device.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _abi as A
from ._abi import check

_DT = {torch.float32: A.NYS_F32, torch.float64: A.NYS_F64, torch.bfloat16: A.NYS_BF16}
_TORCH = {A.NYS_F32: torch.float32, A.NYS_F64: torch.float64, A.NYS_BF16: torch.bfloat16}


def _lib():
    return A.load()


def _ptr(t: torch.Tensor) -> int:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def dtype_code(t: torch.Tensor) -> int:
    try:
        return _DT[t.dtype]
    except KeyError:
        raise ValueError(f"unsupported dtype {t.dtype}") from None


class Context:
    """nys_ctx: device, stream and workspace of the library."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        lib = _lib()
        self.device = device
        s = stream if stream is not None else torch.cuda.current_stream(device)
        self._stream = s
        h = C.c_void_p()
        check(lib.nys_create(C.byref(h), device, C.c_void_p(s.cuda_stream)))
        self.h = h

    def set_stream(self, stream: torch.cuda.Stream):
        self._stream = stream
        check(_lib().nys_set_stream(self.h, C.c_void_p(stream.cuda_stream)), self.h)

    @property
    def stream(self):
        return self._stream

    def sync(self):
        check(_lib().nys_sync(self.h), self.h)

    def reserve(self, nbytes: int):
        check(_lib().nys_reserve(self.h, nbytes), self.h)

    def l2_persist(self, t: torch.Tensor | None, hit_ratio: float = 1.0):
        """Keep tensor t resident in L2 for this context's stream (None clears)."""
        if t is None:
            check(_lib().nys_l2_persist(self.h, None, 0, 0.0), self.h)
        else:
            check(_lib().nys_l2_persist(self.h, _ptr(t), t.numel() * t.element_size(), hit_ratio), self.h)

    def launches(self) -> int:
        n = C.c_int64()
        check(_lib().nys_launch_count(self.h, C.byref(n)), self.h)
        return n.value

    def set_dual_stop(self, on: bool = True):
        """Exact early stop of the mixed-norm dual iteration (bit-identical results)."""
        check(_lib().nys_set_dual_stop(self.h, int(bool(on))), self.h)

    def dual_steps_skipped(self) -> int:
        n = C.c_int64()
        check(_lib().nys_dual_steps_skipped(self.h, C.byref(n)), self.h)
        return n.value

    def last_error(self) -> str:
        return _lib().nys_last_error(self.h).decode()

    def close(self):
        if getattr(self, "h", None):
            _lib().nys_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    """nys_op: blur, blur + decimation, parallel-beam or fan-beam ray transform."""

    def __init__(self, ctx: Context, kind: str, n1: int, n2: int, dtype=torch.float32, kernel=None,
                 decim: int = 1, n_angles: int = 0, n_bins: int = 0, angle_span: float | None = None,
                 haar_levels: int = 0, wavelet: str = "haar", src_dist: float = 0.0, det_dist: float = 0.0,
                 det_spacing: float = 1.0):
        lib = _lib()
        self.ctx, self.kind, self.n1, self.n2, self.dtype = ctx, kind, n1, n2, dtype
        if angle_span is None:
            angle_span = 2.0 * math.pi if kind == "fanbeam" else math.pi
        d = A.nys_op_desc()
        d.kind = {"blur": A.NYS_OP_BLUR, "blur_decim": A.NYS_OP_BLUR_DECIM, "radon": A.NYS_OP_RADON,
                  "fanbeam": A.NYS_OP_FANBEAM}[kind]
        d.dtype = _DT[dtype]
        d.n1, d.n2 = n1, n2
        self._kernel = None
        if kernel is not None:
            k = np.ascontiguousarray(np.asarray(kernel, dtype=np.float64))
            self._kernel = k
            d.kernel = k.ctypes.data_as(C.POINTER(C.c_double))
            d.kh, d.kw = k.shape
        d.decim = decim
        d.n_angles, d.n_bins, d.angle_span = n_angles, n_bins, angle_span
        d.haar_levels = haar_levels
        d.wavelet = {"haar": A.NYS_WAVELET_HAAR, "db4": A.NYS_WAVELET_DB4}[wavelet]
        d.src_dist, d.det_dist, d.det_spacing = src_dist, det_dist, det_spacing
        h = C.c_void_p()
        check(lib.nys_op_create(ctx.h, C.byref(d), C.byref(h)), ctx.h)
        self.h = h
        N, M = C.c_int64(), C.c_int64()
        check(lib.nys_op_sizes(h, C.byref(N), C.byref(M)))
        self.N, self.M = N.value, M.value
        if kind == "blur":
            self.meas_shape = (n1, n2)
        elif kind == "blur_decim":
            self.meas_shape = (n1 // decim, n2 // decim)
        else:
            self.meas_shape = (n_angles, n_bins)

    def autotune(self, batch: int = 1) -> int:
        """Pick the fastest launch variant for `batch` images (synchronises)."""
        c = C.c_int()
        check(_lib().nys_op_autotune(self.h, batch, C.byref(c)), self.ctx.h)
        return c.value

    def set_kernel(self, kernel):
        """Replace the blur kernel (same shape; host copy, synchronises)."""
        k = np.ascontiguousarray(np.asarray(kernel, dtype=np.float64))
        check(_lib().nys_op_set_kernel(self.h, k.ctypes.data_as(C.POINTER(C.c_double)), k.shape[0], k.shape[1]),
              self.ctx.h)
        self._kernel = k

    def close(self):
        if getattr(self, "h", None):
            _lib().nys_op_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _batch(t: torch.Tensor, per: int) -> int:
    if t.numel() % per:
        raise ValueError(f"tensor of {t.numel()} elements is not a batch of {per}")
    return t.numel() // per


def op_apply(op: Operator, x: torch.Tensor, y: torch.Tensor | None = None) -> torch.Tensor:
    b = _batch(x, op.N)
    if y is None:
        y = torch.empty((b,) + op.meas_shape, dtype=x.dtype, device=x.device)
    if x.dtype != op.dtype or y.dtype != op.dtype or _batch(y, op.M) != b:
        raise ValueError("op_apply: dtype or size mismatch")
    check(_lib().op_apply(op.h, _ptr(x), _ptr(y), b), op.ctx.h)
    return y


def op_adjoint(op: Operator, y: torch.Tensor, x: torch.Tensor | None = None) -> torch.Tensor:
    b = _batch(y, op.M)
    if x is None:
        x = torch.empty((b, op.n1, op.n2), dtype=y.dtype, device=y.device)
    if x.dtype != op.dtype or y.dtype != op.dtype or _batch(x, op.N) != b:
        raise ValueError("op_adjoint: dtype or size mismatch")
    check(_lib().op_adjoint(op.h, _ptr(y), _ptr(x), b), op.ctx.h)
    return x


def op_normal(op: Operator, x: torch.Tensor, y: torch.Tensor | None = None) -> torch.Tensor:
    b = _batch(x, op.N)
    if y is None:
        y = torch.empty((b, op.n1, op.n2), dtype=x.dtype, device=x.device)
    if x.dtype != op.dtype or y.dtype != op.dtype or _batch(y, op.N) != b:
        raise ValueError("op_normal: dtype or size mismatch")
    check(_lib().op_normal(op.h, _ptr(x), _ptr(y), b), op.ctx.h)
    return y


def op_haar(op: Operator, x: torch.Tensor, inverse: bool = False, out: torch.Tensor | None = None) -> torch.Tensor:
    b = _batch(x, op.N)
    if out is None:
        out = torch.empty_like(x)
    if out.data_ptr() == x.data_ptr():
        raise ValueError("op_haar: in-place transform is not supported")
    check(_lib().op_haar(op.h, _ptr(x), _ptr(out), b, int(inverse)), op.ctx.h)
    return out


def nys_sketch(ctx: Context, op: Operator, ell: int, seed: int, phi: str = "ata",
               store_dtype=None, out=None) -> tuple[torch.Tensor, torch.Tensor]:
    """Algorithm 1 steps 1-2: returns (Omega, Y), each (ell, n1, n2)."""
    sd = store_dtype or op.dtype
    dev = torch.device("cuda", ctx.device)
    if out is not None:
        Om, Y = out
        if Om.dtype != sd or Y.dtype != sd or Om.numel() != ell * op.N or Y.numel() != ell * op.N:
            raise ValueError("nys_sketch: output buffers do not match")
    else:
        Om = torch.empty((ell, op.n1, op.n2), dtype=sd, device=dev)
        Y = torch.empty_like(Om)
    kind = {"ata": A.NYS_PHI_ATA, "w_ata_wt": A.NYS_PHI_W_ATA_WT}[phi]
    check(_lib().nys_sketch(ctx.h, op.h, kind, ell, seed, _DT[sd], _ptr(Om), _ptr(Y)), ctx.h)
    return Om, Y


def nys_sketch_cols(ctx: Context, op: Operator, ell: int, j0: int, j1: int, seed: int, phi: str = "ata",
                    store_dtype=None) -> tuple[torch.Tensor, torch.Tensor]:
    """Columns j0..j1-1 of the ell-column Omega of nys_sketch and Y = Phi Omega
    for them: (Omega_cols, Y_cols), each (j1 - j0, n1, n2)."""
    sd = store_dtype or op.dtype
    dev = torch.device("cuda", ctx.device)
    Om = torch.empty((j1 - j0, op.n1, op.n2), dtype=sd, device=dev)
    Y = torch.empty_like(Om)
    kind = {"ata": A.NYS_PHI_ATA, "w_ata_wt": A.NYS_PHI_W_ATA_WT}[phi]
    check(_lib().nys_sketch_cols(ctx.h, op.h, kind, ell, j0, j1, seed, _DT[sd], _ptr(Om), _ptr(Y)), ctx.h)
    return Om, Y


def nys_factor_gram(ctx: Context, G2: torch.Tensor, ell: int, eps: float, eig_f64: bool = False):
    """Algorithm 1 steps 3-8 at the ell x ell level from the Gram of [Omega | Y]
    (float64 (2 ell, 2 ell) device tensor): returns (W, S_hat, v, retries)
    with U = (Y + v Omega) W."""
    if G2.dtype != torch.float64 or G2.shape != (2 * ell, 2 * ell):
        raise ValueError("nys_factor_gram: G2 must be float64 (2 ell, 2 ell)")
    W = torch.empty((ell, ell), dtype=torch.float64, device=G2.device)
    S = torch.empty((ell,), dtype=torch.float64, device=G2.device)
    v = C.c_double()
    r = C.c_int()
    check(_lib().nys_factor_gram(ctx.h, _ptr(G2.contiguous()), ell, eps, int(eig_f64), _ptr(W), _ptr(S), C.byref(v),
                                 C.byref(r)), ctx.h)
    return W, S, v.value, r.value


class Precond:
    """nys_precond with caller-owned U (ell, N) and S_hat (ell,) tensors."""

    def __init__(self, ctx: Context, N: int, ell: int, dtype=torch.float32):
        dev = torch.device("cuda", ctx.device)
        self.ctx = ctx
        self.U = torch.empty((ell, N), dtype=dtype, device=dev)
        self.S_hat = torch.empty((ell,), dtype=torch.float64, device=dev)
        self.s = A.nys_precond()
        self.s.U = _ptr(self.U)
        self.s.S_hat = _ptr(self.S_hat)
        self.s.N = N
        self.s.ell = ell
        self.s.dtype = _DT[dtype]
        self.s.mu = float("nan")

    @property
    def v(self) -> float:
        return self.s.v

    @property
    def chol_retries(self) -> int:
        return self.s.chol_retries

    @property
    def ell_active(self) -> int:
        """Columns with d_i > 0 (the only ones P and P^{-1} read)."""
        return self.s.ell_active

    def setup(self, mu: float = 0.0, sqrt_shift: bool = True):
        check(_lib().nys_precond_setup(self.ctx.h, C.byref(self.s), mu, int(sqrt_shift)), self.ctx.h)

    def import_factor(self, U, S_hat, mu: float = 0.0, sqrt_shift: bool = True):
        """Adopt a factor computed elsewhere (arrays or tensors of shape (ell, N), (ell,))."""
        self.U.copy_(torch.as_tensor(U).reshape(self.U.shape).to(self.U.dtype))
        self.S_hat.copy_(torch.as_tensor(S_hat).reshape(self.S_hat.shape).to(torch.float64))
        check(_lib().nys_precond_import(self.ctx.h, C.byref(self.s), mu, int(sqrt_shift)), self.ctx.h)
        return self

    def import_gram(self, U, S_hat, K: torch.Tensor, mu: float = 0.0, sqrt_shift: bool = True):
        """Adopt this rank's rows U (ell, N_local) of a pixel-sharded factor, with
        K = U^T U summed over the ranks (float64 (ell, ell) device tensor)."""
        self.U.copy_(torch.as_tensor(U).reshape(self.U.shape).to(self.U.dtype))
        self.S_hat.copy_(torch.as_tensor(S_hat).reshape(self.S_hat.shape).to(torch.float64))
        check(_lib().nys_precond_import_gram(self.ctx.h, C.byref(self.s), _ptr(K.contiguous()), mu, int(sqrt_shift)),
              self.ctx.h)
        return self

    def close(self):
        if getattr(self, "s", None) is not None and self.s.priv:
            _lib().nys_precond_release(C.byref(self.s))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nys_factor(ctx: Context, Omega: torch.Tensor, Y: torch.Tensor, eps: float, u_dtype=None,
               pc: Precond | None = None) -> Precond:
    """Algorithm 1 steps 3-8 into a Precond (set up with mu = 0, sqrt heuristic on)."""
    ell = Omega.shape[0]
    N = Omega.numel() // ell
    if Y.shape != Omega.shape or Y.dtype != Omega.dtype:
        raise ValueError("nys_factor: Omega and Y must match")
    if pc is None:
        ud = u_dtype or (torch.float64 if Omega.dtype == torch.float64 else torch.float32)
        pc = Precond(ctx, N, ell, ud)
    check(_lib().nys_factor(ctx.h, _ptr(Omega), _ptr(Y), dtype_code(Omega), N, ell, eps, C.byref(pc.s)), ctx.h)
    return pc


def precond_apply(ctx: Context, pc: Precond, z: torch.Tensor, inverse: bool = True,
                  out: torch.Tensor | None = None) -> torch.Tensor:
    b = _batch(z, pc.s.N)
    if out is None:
        out = torch.empty_like(z)
    check(_lib().precond_apply(ctx.h, C.byref(pc.s), int(inverse), dtype_code(z), _ptr(z), _ptr(out), b), ctx.h)
    return out


def precond_partial(ctx: Context, pc: Precond, z: torch.Tensor) -> torch.Tensor:
    """w = U_r^T z_r for this rank's rows (batch, ell_active); the ranks sum w."""
    b = _batch(z, pc.s.N)
    wdt = torch.float64 if z.dtype == torch.float64 else torch.float32
    w = torch.empty((b, max(pc.ell_active, 1)), dtype=wdt, device=z.device)
    check(_lib().precond_partial(ctx.h, C.byref(pc.s), dtype_code(z), _ptr(z), _ptr(w), b), ctx.h)
    return w


def precond_finish(ctx: Context, pc: Precond, w: torch.Tensor, z: torch.Tensor, inverse: bool = True,
                   out: torch.Tensor | None = None) -> torch.Tensor:
    """This rank's rows of P^{-1} z (or P z) from the summed w."""
    b = _batch(z, pc.s.N)
    if out is None:
        out = torch.empty_like(z)
    check(_lib().precond_finish(ctx.h, C.byref(pc.s), int(inverse), dtype_code(z), _ptr(w.contiguous()), _ptr(z),
                                _ptr(out), b), ctx.h)
    return out


def prox_wavelet(ctx: Context, pc: Precond | None, tau: float, s: torch.Tensor, gamma: torch.Tensor | None = None,
                 out: torch.Tensor | None = None):
    if out is None:
        out = torch.empty_like(s)
    info = A.nys_prox_info()
    pcs = C.byref(pc.s) if pc is not None else None
    g = _ptr(gamma) if gamma is not None else None
    check(_lib().prox_wavelet(ctx.h, pcs, tau, dtype_code(s), s.numel(), _ptr(s), _ptr(out), g, C.byref(info)),
          ctx.h)
    return out, dict(iterations=info.iterations, converged=bool(info.converged), residual=info.residual)


def _prox_dual(fn, G, ctx, pc, lam_bar, n_inner, s, Q=None, out=None):
    n1, n2 = s.shape[-2:]
    if Q is None:
        Q = torch.zeros((G, n1, n2), dtype=s.dtype, device=s.device)
    if out is None:
        out = torch.empty_like(s)
    pcs = C.byref(pc.s) if pc is not None else None
    check(fn(ctx.h, pcs, lam_bar, n_inner, dtype_code(s), n1, n2, _ptr(s), _ptr(out), _ptr(Q)), ctx.h)
    return out, Q


def prox_tv(ctx, pc, lam_bar, n_inner, s, Q=None, out=None):
    return _prox_dual(_lib().prox_tv, 2, ctx, pc, lam_bar, n_inner, s, Q, out)


def prox_hs(ctx, pc, lam_bar, n_inner, s, Q=None, out=None):
    return _prox_dual(_lib().prox_hs, 3, ctx, pc, lam_bar, n_inner, s, Q, out)


REGS = {"wavelet": A.NYS_REG_WAVELET, "tv": A.NYS_REG_TV, "hs": A.NYS_REG_HS, "isotv": A.NYS_REG_ISOTV,
        "hs2": A.NYS_REG_HS2, "hsinf": A.NYS_REG_HSINF}


def prox_mixed(ctx, pc, reg: str, lam_bar, n_inner, s, Q=None, out=None):
    """Dual APG prox for any mixed-norm regulariser ("tv", "isotv", "hs", "hs2", "hsinf")."""
    code = REGS[reg]
    fn = lambda *a: _lib().prox_mixed(a[0], a[1], code, *a[2:])
    return _prox_dual(fn, 2 if reg in ("tv", "isotv") else 3, ctx, pc, lam_bar, n_inner, s, Q, out)


class Solver:
    """nys_solver: Algorithm 3 (WAPG; plain APG when pc is None)."""

    def __init__(self, ctx: Context, op: Operator, y: torch.Tensor, reg: str, lam: float, pc: Precond | None = None,
                 fit: str = "l2", huber_delta: float = 0.0, alpha: float = 0.0, n_inner: int = 20,
                 power_iters: int = 50, power_seed: int = 7, use_graph: bool = True):
        d = A.nys_solver_desc()
        d.reg = REGS[reg]
        d.fit = {"l2": A.NYS_FIT_L2, "huber": A.NYS_FIT_HUBER}[fit]
        d.lambda_ = lam
        d.huber_delta = huber_delta
        d.alpha = alpha
        d.n_inner = n_inner
        d.power_iters = power_iters
        d.power_seed = power_seed
        d.no_graph = 0 if use_graph else 1
        self.ctx, self.op, self.pc = ctx, op, pc
        h = C.c_void_p()
        pcs = C.byref(pc.s) if pc is not None else None
        check(_lib().nys_solver_create(ctx.h, op.h, C.byref(d), _ptr(y.contiguous()), pcs, C.byref(h)), ctx.h)
        self.h = h

    def step(self, n: int = 1):
        check(_lib().pgd_step(self.h, n), self.ctx.h)

    def reset(self):
        check(_lib().nys_solver_reset(self.h), self.ctx.h)

    def restart(self, reestimate_alpha: bool = True):
        check(_lib().nys_solver_restart(self.h, int(reestimate_alpha)), self.ctx.h)

    def set_data(self, y: torch.Tensor):
        check(_lib().nys_solver_set_data(self.h, _ptr(y)), self.ctx.h)

    def objective(self) -> float:
        F = C.c_double()
        check(_lib().nys_solver_objective(self.h, C.byref(F)), self.ctx.h)
        return F.value

    @property
    def alpha(self) -> float:
        a = C.c_double()
        check(_lib().nys_solver_alpha(self.h, C.byref(a)), self.ctx.h)
        return a.value

    def x(self, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.op.n1, self.op.n2), dtype=self.op.dtype,
                              device=torch.device("cuda", self.ctx.device))
        check(_lib().nys_solver_get_x(self.h, _ptr(out)), self.ctx.h)
        return out

    def close(self):
        if getattr(self, "h", None):
            _lib().nys_solver_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class IRM:
    """nys_irm: Algorithm 2 (IRM for l_p - l_q, L = first differences) with
    CG, preconditioned by the on-the-fly Nystrom preconditioner when ell > 0."""

    def __init__(self, ctx: Context, op: Operator, y: torch.Tensor, p: float, q: float, lam: float,
                 eps: float = 1e-4, ell: int = 0, store_dtype=torch.bfloat16, seed: int = 0,
                 cg_tol: float = 1e-4, cg_max: int = 1000):
        d = A.nys_irm_desc()
        d.p, d.q, d.lambda_, d.eps = p, q, lam, eps
        d.ell = ell
        d.store_dtype = _DT[torch.float64 if op.dtype == torch.float64 else store_dtype]
        d.seed, d.cg_tol, d.cg_max = seed, cg_tol, cg_max
        self.ctx, self.op = ctx, op
        self._y = y.contiguous()
        h = C.c_void_p()
        check(_lib().nys_irm_create(ctx.h, op.h, C.byref(d), _ptr(self._y), C.byref(h)), ctx.h)
        self.h = h

    def step(self) -> dict:
        info = A.nys_irm_info()
        check(_lib().nys_irm_step(self.h, C.byref(info)), self.ctx.h)
        return {"cg_iters": info.cg_iters, "residual": info.residual, "rel_change": info.rel_change}

    def reset(self):
        check(_lib().nys_irm_reset(self.h), self.ctx.h)

    def x(self) -> torch.Tensor:
        out = torch.empty((self.op.n1, self.op.n2), dtype=self.op.dtype, device=torch.device("cuda", self.ctx.device))
        check(_lib().nys_irm_get_x(self.h, _ptr(out)), self.ctx.h)
        return out

    def close(self):
        if getattr(self, "h", None):
            _lib().nys_irm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pgd_step(solver: Solver, n: int = 1):
    solver.step(n)


class Unroll:
    """nys_unroll: K unrolled TV-regularised Algorithm 3 iterations with a
    hand-written reverse pass (gradients with respect to lambda and the blur
    kernel; P and alpha fixed)."""

    def __init__(self, ctx: Context, op: Operator, lam: float, alpha: float, K: int, n_inner: int = 20,
                 ckpt_every: int = 10, pc: Precond | None = None):
        d = A.nys_unroll_desc()
        d.lambda_, d.alpha, d.K, d.n_inner, d.ckpt_every = lam, alpha, K, n_inner, ckpt_every
        self.ctx, self.op, self.pc, self.lam = ctx, op, pc, lam
        h = C.c_void_p()
        pcs = C.byref(pc.s) if pc is not None else None
        check(_lib().nys_unroll_create(ctx.h, op.h, pcs, C.byref(d), C.byref(h)), ctx.h)
        self.h = h
        self.ntaps = op._kernel.size if op.kind == "blur" else 0

    def set_lambda(self, lam: float):
        check(_lib().nys_unroll_set_lambda(self.h, lam), self.ctx.h)
        self.lam = lam

    def forward(self, y: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.op.n1, self.op.n2), dtype=self.op.dtype, device=y.device)
        check(_lib().nys_unroll_forward(self.h, _ptr(y.contiguous()), _ptr(out)), self.ctx.h)
        return out

    def backward(self, xbar: torch.Tensor):
        """(d<xbar, x>/d lambda as a float64 0-d tensor, d<xbar, x>/dh as a
        float64 (kh, kw) tensor or None) on the device."""
        g = torch.empty(1 + self.ntaps, dtype=torch.float64, device=xbar.device)
        check(_lib().nys_unroll_backward(self.h, _ptr(xbar.contiguous()), _ptr(g)), self.ctx.h)
        dh = g[1:].reshape(self.op._kernel.shape) if self.ntaps else None
        return g[0], dh

    def close(self):
        if getattr(self, "h", None):
            _lib().nys_unroll_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nys_gram(ctx: Context, A: torch.Tensor, B: torch.Tensor, path: int = 0) -> torch.Tensor:
    """A^T B (float64, p x q) for A: (p, N), B: (q, N) stacks of columns."""
    p, q = A.shape[0], B.shape[0]
    N = A.numel() // p
    if A.dtype != B.dtype or B.numel() // q != N:
        raise ValueError("nys_gram: operands do not match")
    C = torch.empty((p, q), dtype=torch.float64, device=A.device)
    check(_lib().nys_gram(ctx.h, dtype_code(A), _ptr(A), p, _ptr(B), q, N, _ptr(C), path), ctx.h)
    return C


def nys_tall_gemm(ctx: Context, A: torch.Tensor, A2: torch.Tensor | None, alpha: float, W: torch.Tensor,
                  out_dtype=None, path: int = 0) -> torch.Tensor:
    """(A + alpha A2) W for A, A2: (k, N) stacks of columns, W: (k, q) float64 -> (q, N)."""
    k = A.shape[0]
    N = A.numel() // k
    q = W.shape[1]
    od = out_dtype or A.dtype
    out = torch.empty((q, N), dtype=od, device=A.device)
    Wd = W.to(torch.float64).contiguous()
    check(_lib().nys_tall_gemm(ctx.h, dtype_code(A), _ptr(A), _ptr(A2) if A2 is not None else None, alpha, N, k,
                               _ptr(Wd), q, _DT[od], _ptr(out), path), ctx.h)
    return out


def nys_rel_err(ctx: Context, a: torch.Tensor, b: torch.Tensor | None) -> float:
    out = C.c_double()
    check(_lib().nys_rel_err(ctx.h, dtype_code(a), a.numel(), _ptr(a), _ptr(b) if b is not None else None,
                             C.byref(out)), ctx.h)
    return out.value


class Batch:
    """nys_batch: several Unroll handles (each on its own Context with its own
    stream) replayed as one CUDA graph for the forward and one for the
    reverse pass.  ys, xs, xbars are per-item device tensors fixed for the
    life of the batch; grads are allocated here (float64, 1 + kh kw each)."""

    def __init__(self, ctx: Context, unrolls: list, ys: list, xs: list, xbars: list):
        n = len(unrolls)
        self.ctx, self.unrolls = ctx, unrolls
        self.ys, self.xs, self.xbars = ys, xs, xbars
        self.grads = [torch.zeros(1 + u.ntaps, dtype=torch.float64, device=torch.device("cuda", ctx.device))
                      for u in unrolls]
        arr = lambda vals: (C.c_void_p * n)(*vals)
        h = C.c_void_p()
        check(_lib().nys_batch_create(ctx.h, n, arr([u.h.value for u in unrolls]),
                                      arr([u.ctx.h.value for u in unrolls]), arr([_ptr(t) for t in ys]),
                                      arr([_ptr(t) for t in xs]), arr([_ptr(t) for t in xbars]),
                                      arr([_ptr(t) for t in self.grads]), C.byref(h)), ctx.h)
        self.h = h

    def forward(self):
        check(_lib().nys_batch_forward(self.h), self.ctx.h)

    def backward(self):
        check(_lib().nys_batch_backward(self.h), self.ctx.h)

    def close(self):
        if getattr(self, "h", None):
            _lib().nys_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
