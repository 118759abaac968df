"""ctypes declarations of the C ABI in include/nys.h.

Marshalling only: every computation happens in libnys.so.  Loading fails
loudly when the library is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libnys.so")

NYS_OK, NYS_EINVAL, NYS_ENOMEM, NYS_ECUDA, NYS_ENOTSPD = 0, 1, 2, 3, 4
NYS_EDEGENERATE, NYS_ENONFINITE, NYS_ETIMEOUT, NYS_ENOCONV = 5, 6, 7, 8
NYS_F32, NYS_F64, NYS_BF16 = 0, 1, 2
NYS_OP_BLUR, NYS_OP_BLUR_DECIM, NYS_OP_RADON, NYS_OP_FANBEAM = 0, 1, 2, 3
NYS_PHI_ATA, NYS_PHI_W_ATA_WT = 0, 1
NYS_REG_WAVELET, NYS_REG_TV, NYS_REG_HS, NYS_REG_ISOTV, NYS_REG_HS2, NYS_REG_HSINF = 0, 1, 2, 3, 4, 5
NYS_WAVELET_HAAR, NYS_WAVELET_DB4 = 0, 1
NYS_FIT_L2, NYS_FIT_HUBER = 0, 1

CODE_NAMES = {0: "NYS_OK", 1: "NYS_EINVAL", 2: "NYS_ENOMEM", 3: "NYS_ECUDA", 4: "NYS_ENOTSPD",
              5: "NYS_EDEGENERATE", 6: "NYS_ENONFINITE", 7: "NYS_ETIMEOUT", 8: "NYS_ENOCONV"}


class nys_op_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("dtype", C.c_int), ("n1", C.c_int), ("n2", C.c_int),
                ("kernel", C.POINTER(C.c_double)), ("kh", C.c_int), ("kw", C.c_int), ("decim", C.c_int),
                ("n_angles", C.c_int), ("n_bins", C.c_int), ("angle_span", C.c_double),
                ("haar_levels", C.c_int), ("wavelet", C.c_int), ("src_dist", C.c_double),
                ("det_dist", C.c_double), ("det_spacing", C.c_double)]


class nys_precond(C.Structure):
    _fields_ = [("U", C.c_void_p), ("S_hat", C.c_void_p), ("N", C.c_int64), ("ell", C.c_int),
                ("dtype", C.c_int), ("v", C.c_double), ("chol_retries", C.c_int), ("s_first", C.c_double),
                ("s_last", C.c_double), ("mu", C.c_double), ("sqrt_shift", C.c_int), ("ell_active", C.c_int),
                ("priv", C.c_void_p)]


class nys_prox_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("residual", C.c_double)]


class nys_irm_desc(C.Structure):
    _fields_ = [("p", C.c_double), ("q", C.c_double), ("lambda_", C.c_double), ("eps", C.c_double),
                ("ell", C.c_int), ("store_dtype", C.c_int), ("seed", C.c_uint64), ("cg_tol", C.c_double),
                ("cg_max", C.c_int)]


class nys_irm_info(C.Structure):
    _fields_ = [("cg_iters", C.c_int), ("residual", C.c_double), ("rel_change", C.c_double)]


class nys_solver_desc(C.Structure):
    _fields_ = [("reg", C.c_int), ("fit", C.c_int), ("lambda_", C.c_double), ("huber_delta", C.c_double),
                ("alpha", C.c_double), ("n_inner", C.c_int), ("power_iters", C.c_int),
                ("power_seed", C.c_uint64), ("no_graph", C.c_int)]


class nys_unroll_desc(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("alpha", C.c_double), ("K", C.c_int), ("n_inner", C.c_int),
                ("ckpt_every", C.c_int)]


vp = C.c_void_p
i32 = C.c_int
i64 = C.c_int64
f64 = C.c_double

# name: (restype, argtypes)
PROTOTYPES = {
    "nys_create": (i32, [C.POINTER(vp), i32, vp]),
    "nys_destroy": (i32, [vp]),
    "nys_set_stream": (i32, [vp, vp]),
    "nys_sync": (i32, [vp]),
    "nys_last_error": (C.c_char_p, [vp]),
    "nys_reserve": (i32, [vp, C.c_size_t]),
    "nys_version": (C.c_char_p, []),
    "nys_launch_count": (i32, [vp, C.POINTER(i64)]),
    "nys_set_dual_stop": (i32, [vp, i32]),
    "nys_dual_steps_skipped": (i32, [vp, C.POINTER(i64)]),
    "nys_l2_persist": (i32, [vp, vp, C.c_size_t, f64]),
    "nys_op_create": (i32, [vp, C.POINTER(nys_op_desc), C.POINTER(vp)]),
    "nys_op_destroy": (i32, [vp]),
    "nys_op_sizes": (i32, [vp, C.POINTER(i64), C.POINTER(i64)]),
    "nys_op_set_kernel": (i32, [vp, C.POINTER(C.c_double), i32, i32]),
    "nys_op_autotune": (i32, [vp, i32, C.POINTER(i32)]),
    "op_apply": (i32, [vp, vp, vp, i32]),
    "op_adjoint": (i32, [vp, vp, vp, i32]),
    "op_normal": (i32, [vp, vp, vp, i32]),
    "op_haar": (i32, [vp, vp, vp, i32, i32]),
    "nys_sketch": (i32, [vp, vp, i32, i32, C.c_uint64, i32, vp, vp]),
    "nys_sketch_cols": (i32, [vp, vp, i32, i32, i32, i32, C.c_uint64, i32, vp, vp]),
    "nys_factor_gram": (i32, [vp, vp, i32, f64, i32, vp, vp, C.POINTER(f64), C.POINTER(i32)]),
    "nys_precond_import_gram": (i32, [vp, C.POINTER(nys_precond), vp, f64, i32]),
    "precond_partial": (i32, [vp, C.POINTER(nys_precond), i32, vp, vp, i32]),
    "precond_finish": (i32, [vp, C.POINTER(nys_precond), i32, i32, vp, vp, vp, i32]),
    "nys_factor": (i32, [vp, vp, vp, i32, i64, i32, f64, C.POINTER(nys_precond)]),
    "nys_precond_release": (i32, [C.POINTER(nys_precond)]),
    "nys_precond_setup": (i32, [vp, C.POINTER(nys_precond), f64, i32]),
    "nys_precond_import": (i32, [vp, C.POINTER(nys_precond), f64, i32]),
    "precond_apply": (i32, [vp, C.POINTER(nys_precond), i32, i32, vp, vp, i32]),
    "precond_apply_noalloc": (i32, [vp, C.POINTER(nys_precond), i32, i32, vp, vp, i32]),
    "prox_wavelet": (i32, [vp, C.POINTER(nys_precond), f64, i32, i64, vp, vp, vp, C.POINTER(nys_prox_info)]),
    "prox_tv": (i32, [vp, C.POINTER(nys_precond), f64, i32, i32, i32, i32, vp, vp, vp]),
    "prox_hs": (i32, [vp, C.POINTER(nys_precond), f64, i32, i32, i32, i32, vp, vp, vp]),
    "prox_mixed": (i32, [vp, C.POINTER(nys_precond), i32, f64, i32, i32, i32, i32, vp, vp, vp]),
    "nys_solver_create": (i32, [vp, vp, C.POINTER(nys_solver_desc), vp, C.POINTER(nys_precond), C.POINTER(vp)]),
    "nys_irm_create": (i32, [vp, vp, C.POINTER(nys_irm_desc), vp, C.POINTER(vp)]),
    "nys_irm_step": (i32, [vp, C.POINTER(nys_irm_info)]),
    "nys_irm_get_x": (i32, [vp, vp]),
    "nys_irm_reset": (i32, [vp]),
    "nys_irm_destroy": (i32, [vp]),
    "nys_solver_destroy": (i32, [vp]),
    "pgd_step": (i32, [vp, i32]),
    "nys_solver_reset": (i32, [vp]),
    "nys_solver_restart": (i32, [vp, i32]),
    "nys_solver_set_data": (i32, [vp, vp]),
    "nys_solver_get_x": (i32, [vp, vp]),
    "nys_solver_alpha": (i32, [vp, C.POINTER(f64)]),
    "nys_solver_objective": (i32, [vp, C.POINTER(f64)]),
    "nys_unroll_create": (i32, [vp, vp, C.POINTER(nys_precond), C.POINTER(nys_unroll_desc), C.POINTER(vp)]),
    "nys_unroll_destroy": (i32, [vp]),
    "nys_unroll_forward": (i32, [vp, vp, vp]),
    "nys_unroll_backward": (i32, [vp, vp, vp]),
    "nys_unroll_set_lambda": (i32, [vp, f64]),
    "nys_batch_create": (i32, [vp, i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                               C.POINTER(vp), C.POINTER(vp)]),
    "nys_batch_forward": (i32, [vp]),
    "nys_batch_backward": (i32, [vp]),
    "nys_batch_destroy": (i32, [vp]),
    "nys_rel_err": (i32, [vp, i32, i64, vp, vp, C.POINTER(f64)]),
    "nys_gram": (i32, [vp, i32, vp, i32, vp, i32, i64, vp, i32]),
    "nys_tall_gemm": (i32, [vp, i32, vp, vp, f64, i64, i32, vp, i32, i32, vp, i32]),
}


class NysError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{CODE_NAMES.get(code, code)}: {msg}")
        self.code = code


_LIB = None


def load(path: str | None = None) -> C.CDLL:
    """Load libnys.so (once).  Raises if it is missing: there is no fallback."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = path or os.environ.get("NYS_LIB", LIB_PATH)
    if not os.path.exists(p):
        raise ImportError(f"libnys.so not found at {p}: build it with "
                          f"`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(p)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def check(code: int, ctx=None):
    if code != NYS_OK:
        lib = load()
        msg = lib.nys_last_error(ctx).decode() if ctx else lib.nys_last_error(None).decode()
        raise NysError(code, msg)
