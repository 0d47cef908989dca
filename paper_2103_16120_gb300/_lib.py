"""ctypes declarations of the C ABI in include/sw_elliptic.h.

Loading fails loudly (ImportError) when libsw_elliptic.so has not been built:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsw_elliptic.so")

SW_OK, SW_ERR_INVALID_ARG, SW_ERR_CUDA, SW_ERR_OOM, SW_ERR_NOT_CONVERGED, SW_ERR_BREAKDOWN, \
    SW_ERR_NONFINITE, SW_ERR_TIMEOUT, SW_ERR_INTERNAL = range(9)
STATUS_NAMES = {0: "SW_OK", 1: "SW_ERR_INVALID_ARG", 2: "SW_ERR_CUDA", 3: "SW_ERR_OOM",
                4: "SW_ERR_NOT_CONVERGED", 5: "SW_ERR_BREAKDOWN", 6: "SW_ERR_NONFINITE",
                7: "SW_ERR_TIMEOUT", 8: "SW_ERR_INTERNAL"}
SW_PREC_FP64, SW_PREC_MIXED_FP16, SW_PREC_MIXED_BF16, SW_PREC_FP32 = range(4)
SW_PC_NONE, SW_PC_DIAG, SW_PC_DIAG_RICHARDSON, SW_PC_SI_RICHARDSON, SW_PC_LEARNED = range(5)

# every symbol the header declares (checked by the CPU test-suite)
EXPORTS = (
    "sw_solve_opts_default", "sw_grid_create", "sw_grid_destroy", "sw_grid_workspace_bytes",
    "sw_grid_attach_workspace", "sw_elliptic_set_coeffs", "sw_grid_set_eta", "sw_grid_get_eta",
    "sw_operator_apply", "sw_precond_apply", "sw_gcr_solve", "sw_ensemble_solve", "sw_gcr_solve_noalloc",
    "sw_last_error", "sw_model_create", "sw_model_destroy", "sw_model_set_params", "sw_model_get_params",
    "sw_model_features", "sw_model_forward", "sw_model_loss_grad", "sw_model_train_step", "sw_model_apply",
    "sw_model_target", "sw_ensemble_solve_async", "sw_debug_barrier",
    "sw_swe_create", "sw_swe_destroy", "sw_swe_set_state", "sw_swe_set_history", "sw_swe_get_state",
    "sw_swe_explicit", "sw_swe_step", "sw_split_refresh", "sw_split_residual",
)
SW_MODEL_PARAMS = 158369
SW_NOALLOC_SCRATCH_BYTES = 16 << 20


class SolveOpts(C.Structure):
    _fields_ = [("k", C.c_int), ("tol", C.c_double), ("max_iters", C.c_int), ("min_iters", C.c_int),
                ("pc", C.c_int), ("n_richardson", C.c_int), ("eta", C.c_double), ("omega", C.c_double),
                ("prec", C.c_int), ("pole_band_rows", C.c_int), ("ru_every", C.c_int),
                ("threads_per_row", C.c_int),
                ("res_history", C.c_void_p), ("row_residual", C.c_void_p),
                ("model", C.c_void_p), ("fb_ratio", C.c_double), ("row_mode", C.c_int),
                ("split_r0", C.c_int)]


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("status", C.c_int),
                ("fallbacks", C.c_int), ("r0_norm", C.c_double), ("R_norm", C.c_double),
                ("true_rel_residual", C.c_double), ("recursive_rel_residual", C.c_double),
                ("eta", C.c_double), ("network_turns", C.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class SweParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("gravity", C.c_double), ("omega", C.c_double)]


class AdamW(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("weight_decay", C.c_double)]


_lib = None


def load() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_2103_16120_gb300.build.build() "
                          "(the solver has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    vp, i, d, st = C.c_void_p, C.c_int, C.c_double, C.c_int
    lib.sw_solve_opts_default.argtypes = [C.POINTER(SolveOpts)]
    lib.sw_solve_opts_default.restype = None
    lib.sw_grid_create.argtypes = [i, i, d, C.POINTER(vp)]
    lib.sw_grid_destroy.argtypes = [vp]
    lib.sw_grid_workspace_bytes.argtypes = [vp, C.POINTER(SolveOpts), C.POINTER(C.c_size_t)]
    lib.sw_grid_attach_workspace.argtypes = [vp, vp, C.c_size_t]
    lib.sw_elliptic_set_coeffs.argtypes = [vp] * 8 + [vp]
    lib.sw_grid_set_eta.argtypes = [vp, d, vp]
    lib.sw_grid_get_eta.argtypes = [vp, C.POINTER(d)]
    lib.sw_operator_apply.argtypes = [vp, i, vp, vp, vp]
    lib.sw_precond_apply.argtypes = [vp, C.POINTER(SolveOpts), vp, vp, vp]
    lib.sw_gcr_solve.argtypes = [vp, C.POINTER(SolveOpts), vp, vp, C.POINTER(SolveStats), vp]
    lib.sw_debug_barrier.argtypes = [i, d]
    lib.sw_ensemble_solve_async.argtypes = [i, C.POINTER(vp), C.POINTER(SolveOpts), C.POINTER(vp),
                                            C.POINTER(vp), vp, vp]
    lib.sw_gcr_solve_noalloc.argtypes = [vp, C.POINTER(SolveOpts), vp, vp, C.POINTER(SolveStats), vp]
    lib.sw_ensemble_solve.argtypes = [i, C.POINTER(vp), C.POINTER(SolveOpts), C.POINTER(vp),
                                      C.POINTER(vp), C.POINTER(SolveStats), vp]
    fp = C.POINTER(C.c_float)
    lib.sw_model_create.argtypes = [C.POINTER(vp)]
    lib.sw_model_destroy.argtypes = [vp]
    lib.sw_model_set_params.argtypes = [vp, vp]
    lib.sw_model_get_params.argtypes = [vp, vp]
    lib.sw_model_features.argtypes = [vp, vp, vp, vp, vp]
    lib.sw_model_forward.argtypes = [vp, i, i, i, vp, vp, vp]
    lib.sw_model_loss_grad.argtypes = [vp, i, i, i, vp, vp, C.POINTER(d), vp, vp]
    lib.sw_model_train_step.argtypes = [vp, i, i, i, vp, vp, C.POINTER(AdamW), C.POINTER(d), vp]
    lib.sw_model_apply.argtypes = [vp, vp, vp, vp, vp]
    lib.sw_model_target.argtypes = [vp, vp, vp, vp, vp, vp]
    del fp
    lib.sw_swe_create.argtypes = [vp, C.POINTER(SweParams), C.POINTER(vp)]
    lib.sw_swe_destroy.argtypes = [vp]
    lib.sw_swe_set_state.argtypes = [vp] * 8 + [vp]
    lib.sw_swe_set_history.argtypes = [vp, vp, vp, vp]
    lib.sw_swe_get_state.argtypes = [vp, vp, vp, vp, vp]
    lib.sw_swe_explicit.argtypes = [vp, vp, C.POINTER(vp), vp, vp]
    lib.sw_swe_step.argtypes = [vp, C.POINTER(SolveOpts), i, C.POINTER(SolveStats), vp]
    lib.sw_last_error.argtypes = []
    lib.sw_last_error.restype = C.c_char_p
    for name in EXPORTS:
        f = getattr(lib, name)
        if name not in ("sw_solve_opts_default", "sw_last_error"):
            f.restype = st
    _lib = lib
    return lib
