"""GB300-native elliptic solver for the semi-implicit shallow-water model on
the longitude/latitude sphere (preconditioned GCR(k), Sec. 2.3).

Thin Python binding of the C ABI (include/sw_elliptic.h): the functions keep
the ABI's names and only marshal arguments -- torch CUDA tensors become device
pointers, the current torch stream becomes the CUDA stream.  Every step of the
solve runs in the library's CUDA kernels; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
from typing import Sequence

from ._lib import (  # noqa: F401
    EXPORTS, SolveOpts, SolveStats, STATUS_NAMES, load,
    SW_OK, SW_ERR_INVALID_ARG, SW_ERR_CUDA, SW_ERR_OOM, SW_ERR_NOT_CONVERGED, SW_ERR_BREAKDOWN,
    SW_ERR_NONFINITE, SW_ERR_TIMEOUT, SW_ERR_INTERNAL,
    SW_PREC_FP64, SW_PREC_MIXED_FP16, SW_PREC_MIXED_BF16, SW_PREC_FP32,
    SW_PC_NONE, SW_PC_DIAG, SW_PC_DIAG_RICHARDSON, SW_PC_SI_RICHARDSON, SW_PC_LEARNED, SW_NOALLOC_SCRATCH_BYTES,
    SW_MODEL_PARAMS, AdamW, SweParams,
)

COEFF_KEYS = ("A11", "A12", "A21", "A22", "B1", "B2", "C")
# outcomes of a solve that are reported in the stats rather than raised
SOLVE_OUTCOMES = (SW_OK, SW_ERR_NOT_CONVERGED, SW_ERR_BREAKDOWN, SW_ERR_NONFINITE)


class SwError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().sw_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status: int, where: str, allowed=(SW_OK,)):
    if status not in allowed:
        raise SwError(status, where)
    return status


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t, dtype=None, shape=None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


def sw_solve_opts_default(**overrides) -> SolveOpts:
    o = SolveOpts()
    load().sw_solve_opts_default(C.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        if k in ("res_history", "row_residual") and v is not None and not isinstance(v, int):
            v = v.data_ptr()
        if k == "model" and isinstance(v, Model):
            v = v.handle.value
        setattr(o, k, v)
    return o


class Grid:
    """Handle of an nx x ny grid (sw_grid); destroyed with the object."""

    def __init__(self, nx: int, ny: int, radius: float = 6.371e6):
        h = C.c_void_p()
        _check(load().sw_grid_create(int(nx), int(ny), float(radius), C.byref(h)), "sw_grid_create")
        self.handle = h
        self.nx, self.ny = int(nx), int(ny)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                load().sw_grid_destroy(h)
            except Exception:
                pass
            self.handle = None


def sw_grid_create(nx: int, ny: int, radius: float = 6.371e6) -> Grid:
    return Grid(nx, ny, radius)


def sw_grid_destroy(g: Grid) -> None:
    if g.handle is not None and g.handle.value:
        _check(load().sw_grid_destroy(g.handle), "sw_grid_destroy")
        g.handle = None


def sw_grid_workspace_bytes(g: Grid, opts: SolveOpts | None = None) -> int:
    n = C.c_size_t()
    _check(load().sw_grid_workspace_bytes(g.handle, C.byref(opts) if opts else None, C.byref(n)),
           "sw_grid_workspace_bytes")
    return n.value


def sw_grid_attach_workspace(g: Grid, buf) -> None:
    ptr = None if buf is None else C.c_void_p(buf.data_ptr())
    nbytes = 0 if buf is None else buf.numel() * buf.element_size()
    _check(load().sw_grid_attach_workspace(g.handle, ptr, nbytes), "sw_grid_attach_workspace")


def sw_elliptic_set_coeffs(g: Grid, A11, A12, A21, A22, B1, B2, C_, stream=None) -> None:
    import torch
    shp = (g.ny, g.nx)
    ptrs = [_ptr(t, torch.float64, shp) for t in (A11, A12, A21, A22, B1, B2, C_)]
    _check(load().sw_elliptic_set_coeffs(g.handle, *ptrs, _stream(stream)), "sw_elliptic_set_coeffs")


def sw_grid_set_eta(g: Grid, eta: float, stream=None) -> None:
    _check(load().sw_grid_set_eta(g.handle, float(eta), _stream(stream)), "sw_grid_set_eta")


def sw_grid_get_eta(g: Grid) -> float:
    v = C.c_double()
    _check(load().sw_grid_get_eta(g.handle, C.byref(v)), "sw_grid_get_eta")
    return v.value


def sw_operator_apply(g: Grid, x, y, stream=None) -> None:
    """y = L(x); FP64 for float64 tensors, FP32 for float32 tensors."""
    import torch
    prec = SW_PREC_FP64 if x.dtype == torch.float64 else SW_PREC_FP32
    dt = torch.float64 if prec == SW_PREC_FP64 else torch.float32
    shp = (g.ny, g.nx)
    _check(load().sw_operator_apply(g.handle, prec, _ptr(x, dt, shp), _ptr(y, dt, shp), _stream(stream)),
           "sw_operator_apply")


def sw_split_refresh(g: Grid, phi, stream=None) -> None:
    """Store Phi_hat = fp32(phi) and its flux derivative parts (Sec. 4.2, Eq. 14)."""
    import torch
    _check(load().sw_split_refresh(g.handle, _ptr(phi, torch.float64, (g.ny, g.nx)), _stream(stream)),
           "sw_split_refresh")


def sw_split_residual(g: Grid, phi, R, r, stream=None) -> None:
    """r = L(phi) - R with L in FP32 by the split form of Eq. 14 (r float32)."""
    import torch
    shp = (g.ny, g.nx)
    _check(load().sw_split_residual(g.handle, _ptr(phi, torch.float64, shp), _ptr(R, torch.float64, shp),
                                    _ptr(r, torch.float32, shp), _stream(stream)), "sw_split_residual")


def sw_precond_apply(g: Grid, opts: SolveOpts, r, q, stream=None) -> None:
    import torch
    dt = torch.float64 if opts.prec == SW_PREC_FP64 else torch.float32
    shp = (g.ny, g.nx)
    _check(load().sw_precond_apply(g.handle, C.byref(opts), _ptr(r, dt, shp), _ptr(q, dt, shp), _stream(stream)),
           "sw_precond_apply")


def sw_gcr_solve(g: Grid, opts: SolveOpts, R, phi, stream=None) -> SolveStats:
    """Solve L(phi) = R in place (phi: first guess in, solution out)."""
    import torch
    shp = (g.ny, g.nx)
    st = SolveStats()
    _check(load().sw_gcr_solve(g.handle, C.byref(opts), _ptr(R, torch.float64, shp),
                               _ptr(phi, torch.float64, shp), C.byref(st), _stream(stream)),
           "sw_gcr_solve", SOLVE_OUTCOMES)
    return st


def sw_ensemble_solve_async(grids: Sequence[Grid], opts: SolveOpts, Rs, phis, stats_dev=None, stream=None) -> None:
    """Enqueue an ensemble solve without synchronising; stats_dev: a device
    buffer of len(grids) * sizeof(SolveStats) bytes (torch uint8) or None;
    read it with stats_from_device."""
    import torch
    n = len(grids)
    hs = (C.c_void_p * n)(*[g.handle.value for g in grids])
    rp = (C.c_void_p * n)(*[_ptr(R, torch.float64, (g.ny, g.nx)).value for g, R in zip(grids, Rs)])
    pp = (C.c_void_p * n)(*[_ptr(p, torch.float64, (g.ny, g.nx)).value for g, p in zip(grids, phis)])
    if stats_dev is not None and stats_dev.numel() < n * C.sizeof(SolveStats):
        raise ValueError("stats_dev too small")
    _check(load().sw_ensemble_solve_async(n, hs, C.byref(opts), rp, pp,
                                          None if stats_dev is None else C.c_void_p(stats_dev.data_ptr()),
                                          _stream(stream)), "sw_ensemble_solve_async")


def stats_buffer(n: int):
    import torch
    return torch.zeros(n * C.sizeof(SolveStats), dtype=torch.uint8, device="cuda")


def stats_from_device(buf, n: int) -> list:
    raw = bytes(buf.cpu().numpy().tobytes())
    arr = (SolveStats * n).from_buffer_copy(raw[: n * C.sizeof(SolveStats)])
    return list(arr)


def sw_gcr_solve_noalloc(g: Grid, opts: SolveOpts, R, phi, stream=None) -> SolveStats:
    """sw_gcr_solve with the work vectors in the library's fixed device scratch
    (no allocation; grids up to SW_NOALLOC_SCRATCH_BYTES of workspace)."""
    import torch
    shp = (g.ny, g.nx)
    st = SolveStats()
    _check(load().sw_gcr_solve_noalloc(g.handle, C.byref(opts), _ptr(R, torch.float64, shp),
                                       _ptr(phi, torch.float64, shp), C.byref(st), _stream(stream)),
           "sw_gcr_solve_noalloc", SOLVE_OUTCOMES)
    return st


def sw_ensemble_solve(grids: Sequence[Grid], opts: SolveOpts, Rs, phis, stream=None) -> list:
    import torch
    n = len(grids)
    hs = (C.c_void_p * n)(*[g.handle.value for g in grids])
    rp = (C.c_void_p * n)(*[_ptr(R, torch.float64, (g.ny, g.nx)).value for g, R in zip(grids, Rs)])
    pp = (C.c_void_p * n)(*[_ptr(p, torch.float64, (g.ny, g.nx)).value for g, p in zip(grids, phis)])
    stats = (SolveStats * n)()
    _check(load().sw_ensemble_solve(n, hs, C.byref(opts), rp, pp, stats, _stream(stream)),
           "sw_ensemble_solve", SOLVE_OUTCOMES)
    return list(stats)


# ---------------------------------------------------------------------------
# learned preconditioner
# ---------------------------------------------------------------------------
class Model:
    """Handle of a learned-preconditioner network (sw_model); destroyed with the object."""

    def __init__(self):
        self.handle = C.c_void_p()
        _check(load().sw_model_create(C.byref(self.handle)), "sw_model_create")

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value:
            try:
                load().sw_model_destroy(self.handle)
            except Exception:
                pass
            self.handle = C.c_void_p()


def sw_model_set_params(m: Model, params) -> None:
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != SW_MODEL_PARAMS:
        raise ValueError(f"expected {SW_MODEL_PARAMS} parameters, got {p.size}")
    _check(load().sw_model_set_params(m.handle, p.ctypes.data), "sw_model_set_params")


def sw_model_get_params(m: Model):
    import numpy as np
    p = np.empty(SW_MODEL_PARAMS, dtype=np.float32)
    _check(load().sw_model_get_params(m.handle, p.ctypes.data), "sw_model_get_params")
    return p


def sw_model_features(m: Model, g: Grid, r, x0, stream=None) -> None:
    import torch
    _check(load().sw_model_features(m.handle, g.handle, _ptr(r, torch.float32, (g.ny, g.nx)),
                                    _ptr(x0, torch.float32, (4, g.ny, g.nx)), _stream(stream)), "sw_model_features")


def sw_model_forward(m: Model, x0, y, stream=None) -> None:
    import torch
    B, _, ny, nx = x0.shape
    _check(load().sw_model_forward(m.handle, B, ny, nx, _ptr(x0, torch.float32, (B, 4, ny, nx)),
                                   _ptr(y, torch.float32, (B, ny, nx)), _stream(stream)), "sw_model_forward")


def sw_model_loss_grad(m: Model, x0, target, want_grad: bool = True, stream=None):
    import numpy as np
    import torch
    B, _, ny, nx = x0.shape
    loss = C.c_double()
    g = np.empty(SW_MODEL_PARAMS, dtype=np.float32) if want_grad else None
    _check(load().sw_model_loss_grad(m.handle, B, ny, nx, _ptr(x0, torch.float32, (B, 4, ny, nx)),
                                     _ptr(target, torch.float32, (B, ny, nx)), C.byref(loss),
                                     g.ctypes.data if g is not None else None, _stream(stream)),
           "sw_model_loss_grad")
    return loss.value, g


def sw_model_train_step(m: Model, x0, target, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                        eps: float = 1e-8, weight_decay: float = 0.0, want_loss: bool = True, stream=None):
    import torch
    B, _, ny, nx = x0.shape
    hp = AdamW(lr, beta1, beta2, eps, weight_decay)
    loss = C.c_double()
    _check(load().sw_model_train_step(m.handle, B, ny, nx, _ptr(x0, torch.float32, (B, 4, ny, nx)),
                                      _ptr(target, torch.float32, (B, ny, nx)), C.byref(hp),
                                      C.byref(loss) if want_loss else None, _stream(stream)),
           "sw_model_train_step")
    return loss.value if want_loss else None


def sw_model_apply(m: Model, g: Grid, r, e, stream=None) -> None:
    import torch
    _check(load().sw_model_apply(m.handle, g.handle, _ptr(r, torch.float32, (g.ny, g.nx)),
                                 _ptr(e, torch.float32, (g.ny, g.nx)), _stream(stream)), "sw_model_apply")


def sw_model_target(m: Model, g: Grid, r, e, y, stream=None) -> None:
    import torch
    shp = (g.ny, g.nx)
    _check(load().sw_model_target(m.handle, g.handle, _ptr(r, torch.float32, shp), _ptr(e, torch.float32, shp),
                                  _ptr(y, torch.float32, shp), _stream(stream)), "sw_model_target")


def sw_debug_barrier(extra_arrivals: int, wait_limit_s: float) -> None:
    _check(load().sw_debug_barrier(int(extra_arrivals), float(wait_limit_s)), "sw_debug_barrier")


# ---------------------------------------------------------------------------
# semi-implicit shallow-water time stepping around the solve (Eqs. 1-10)
# ---------------------------------------------------------------------------
class Swe:
    """Handle of a time stepper on a grid (sw_swe); destroyed with the object.
    Keeps a reference to the grid, which must outlive it."""

    def __init__(self, g: Grid, dt: float, gravity: float = 9.80616, omega: float = 7.292e-5):
        self.grid = g
        self.handle = C.c_void_p()
        p = SweParams(float(dt), float(gravity), float(omega))
        _check(load().sw_swe_create(g.handle, C.byref(p), C.byref(self.handle)), "sw_swe_create")

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value:
            try:
                load().sw_swe_destroy(self.handle)
            except Exception:
                pass
            self.handle = C.c_void_p()


def sw_swe_create(g: Grid, dt: float, gravity: float = 9.80616, omega: float = 7.292e-5) -> Swe:
    return Swe(g, dt, gravity, omega)


def sw_swe_set_state(m: Swe, Phi, Qx, Qy, H0=None, alpha=None, Qbar_x=None, Qbar_y=None, stream=None) -> None:
    import torch
    shp = (m.grid.ny, m.grid.nx)
    ptrs = [_ptr(t, torch.float64, shp) for t in (Phi, Qx, Qy, H0, alpha, Qbar_x, Qbar_y)]
    _check(load().sw_swe_set_state(m.handle, *ptrs, _stream(stream)), "sw_swe_set_state")


def sw_swe_set_history(m: Swe, u_prev, v_prev, stream=None) -> None:
    import torch
    shp = (m.grid.ny, m.grid.nx)
    _check(load().sw_swe_set_history(m.handle, _ptr(u_prev, torch.float64, shp), _ptr(v_prev, torch.float64, shp),
                                     _stream(stream)), "sw_swe_set_history")


def sw_swe_get_state(m: Swe, Phi=None, Qx=None, Qy=None, stream=None) -> None:
    import torch
    shp = (m.grid.ny, m.grid.nx)
    ptrs = [_ptr(t, torch.float64, shp) for t in (Phi, Qx, Qy)]
    _check(load().sw_swe_get_state(m.handle, *ptrs, _stream(stream)), "sw_swe_get_state")


def sw_swe_explicit(m: Swe, phi_star=None, coeffs=None, rhs=None, stream=None) -> None:
    """Steps 1-4 of the next step for the predictor phi_star (None: Phi^n);
    coeffs: None or 7 tensors (A11..C, entries may be None) receiving the
    coefficient fields; rhs: None or a tensor for R'."""
    import torch
    shp = (m.grid.ny, m.grid.nx)
    arr = None
    if coeffs is not None:
        if len(coeffs) != 7:
            raise ValueError("coeffs needs 7 entries")
        arr = (C.c_void_p * 7)(*[None if t is None else _ptr(t, torch.float64, shp).value for t in coeffs])
    _check(load().sw_swe_explicit(m.handle, _ptr(phi_star, torch.float64, shp), arr,
                                  _ptr(rhs, torch.float64, shp), _stream(stream)), "sw_swe_explicit")


def sw_swe_step(m: Swe, opts: SolveOpts, nsteps: int = 1, want_stats: bool = True, stream=None):
    """Advance nsteps steps; returns the list of every solve's SolveStats
    (2 per step: predictor, corrector; synchronising), or None with
    want_stats=False (nothing synchronises)."""
    stats = (SolveStats * (2 * int(nsteps)))() if want_stats else None
    _check(load().sw_swe_step(m.handle, C.byref(opts), int(nsteps), stats, _stream(stream)), "sw_swe_step")
    return list(stats) if want_stats else None
