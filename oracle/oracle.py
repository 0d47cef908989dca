"""ctypes binding of the C oracle (oracle/sw_oracle.c).  Test infrastructure only.

All arrays are float64 numpy arrays of shape (ny, nx), C-contiguous.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sw_oracle.c")
_LIB = os.path.join(_HERE, "libsw_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, IEEE semantics, OpenMP over rows)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int)] + [
        (k, C.POINTER(C.c_double)) for k in ("A11", "A12", "A21", "A22", "B1", "B2", "C")]


class _Opts(C.Structure):
    _fields_ = [("k", C.c_int), ("tol", C.c_double), ("max_iters", C.c_int),
                ("min_iters", C.c_int), ("pc", C.c_int), ("n_rich", C.c_int),
                ("eta", C.c_double), ("omega", C.c_double), ("ru_every", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("status", C.c_int),
                ("r0_norm", C.c_double), ("R_norm", C.c_double),
                ("true_rel_residual", C.c_double), ("recursive_rel_residual", C.c_double),
                ("eta_used", C.c_double)]


_lib = None


def _get():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        pd = C.POINTER(C.c_double)
        P = C.POINTER(_Problem)
        _lib.swo_operator.argtypes = [P, pd, pd]
        _lib.swo_apply_PZ.argtypes = [P, pd, pd]
        _lib.swo_apply_PM.argtypes = [P, pd, pd]
        _lib.swo_diag_L.argtypes = [P, pd]
        _lib.swo_eta_auto.argtypes = [P]
        _lib.swo_eta_auto.restype = C.c_double
        _lib.swo_cyclic_solve.argtypes = [C.c_int, pd, pd, pd, pd, pd]
        _lib.swo_row_T.argtypes = [P, C.c_int, C.c_double, pd, pd, pd]
        _lib.swo_precond.argtypes = [P, C.POINTER(_Opts), C.c_double, pd, pd]
        _lib.swo_gcr.argtypes = [P, C.POINTER(_Opts), pd, pd, C.POINTER(_Stats), pd, pd]
        _lib.swo_gcr.restype = C.c_int
        _lib.swo_round_bits.argtypes = [C.c_double, C.c_int]
        _lib.swo_round_bits.restype = C.c_double
        _lib.swo_set_threads.argtypes = [C.c_int]
        _lib.swo_set_threads.restype = None
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


COEFF_KEYS = ("A11", "A12", "A21", "A22", "B1", "B2", "C")


class Problem:
    """Coefficient fields of Eq. 10 held for the oracle calls."""

    def __init__(self, coeffs: dict):
        self._arrs = {k: np.ascontiguousarray(coeffs[k], dtype=np.float64) for k in COEFF_KEYS}
        ny, nx = self._arrs["C"].shape
        self.nx, self.ny = nx, ny
        self._s = _Problem(nx, ny, *[_ptr(self._arrs[k]) for k in COEFF_KEYS])

    def _new(self):
        return np.zeros((self.ny, self.nx))

    def _x(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        assert x.shape == (self.ny, self.nx)
        return x

    def operator(self, x):
        """L(x), Eq. 10."""
        x = self._x(x); y = self._new()
        _get().swo_operator(C.byref(self._s), _ptr(x), _ptr(y))
        return y

    def apply_PZ(self, x):
        x = self._x(x); y = self._new()
        _get().swo_apply_PZ(C.byref(self._s), _ptr(x), _ptr(y))
        return y

    def apply_PM(self, x):
        x = self._x(x); y = self._new()
        _get().swo_apply_PM(C.byref(self._s), _ptr(x), _ptr(y))
        return y

    def diag_L(self):
        d = self._new()
        _get().swo_diag_L(C.byref(self._s), _ptr(d))
        return d

    def eta_auto(self) -> float:
        return _get().swo_eta_auto(C.byref(self._s))

    def row_T(self, j: int, eta: float):
        sub, diag, sup = (np.zeros(self.nx) for _ in range(3))
        _get().swo_row_T(C.byref(self._s), j, eta, _ptr(sub), _ptr(diag), _ptr(sup))
        return sub, diag, sup

    def precond(self, r, opts: "Opts", eta: float | None = None):
        r = self._x(r); q = self._new()
        if eta is None:
            eta = opts.eta if opts.eta > 0 else self.eta_auto()
        o = opts.to_c()
        _get().swo_precond(C.byref(self._s), C.byref(o), eta, _ptr(r), _ptr(q))
        return q

    def gcr(self, R, opts: "Opts", phi0=None, want_history: bool = False):
        """Preconditioned GCR(k).  Returns (phi, stats dict[, hist, orth])."""
        R = self._x(R)
        phi = self._new() if phi0 is None else self._x(phi0).copy()
        st = _Stats()
        hist = np.full(opts.max_iters + 1, np.nan)
        orth = np.full(max(opts.max_iters, 1), np.nan)
        o = opts.to_c()
        _get().swo_gcr(C.byref(self._s), C.byref(o), _ptr(R), _ptr(phi), C.byref(st),
                       _ptr(hist), _ptr(orth))
        stats = {f: getattr(st, f) for f, _ in _Stats._fields_}
        if want_history:
            return phi, stats, hist[: st.iterations + 1], orth[: st.iterations]
        return phi, stats


@dataclass
class Opts:
    """Solver options; same meaning as the library's sw_solve_opts."""
    k: int = 4
    tol: float = 1e-10
    max_iters: int = 200
    min_iters: int = 0
    pc: int = 3
    n_rich: int = 2
    eta: float = 0.0
    omega: float = 1.0
    ru_every: int = 0

    def to_c(self) -> _Opts:
        return _Opts(self.k, self.tol, self.max_iters, self.min_iters, self.pc,
                     self.n_rich, self.eta, self.omega, self.ru_every)


def cyclic_solve(sub, diag, sup, rhs):
    n = len(diag)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (sub, diag, sup, rhs)]
    x = np.zeros(n)
    _get().swo_cyclic_solve(n, *[_ptr(a) for a in arrs], _ptr(x))
    return x


def set_threads(n: int) -> None:
    """Host threads of the oracle's row loops (results do not depend on it)."""
    _get().swo_set_threads(int(n))


def round_bits(x: float, p: int) -> float:
    return _get().swo_round_bits(float(x), int(p))


def operator_matrix(prob: Problem) -> np.ndarray:
    """Dense matrix of L assembled column by column (brute force, small grids)."""
    n = prob.nx * prob.ny
    M = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n); e[c] = 1.0
        M[:, c] = prob.operator(e.reshape(prob.ny, prob.nx)).ravel()
    return M
