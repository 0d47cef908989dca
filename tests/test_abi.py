"""CPU-only checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/sw_elliptic.h declares, the ctypes mirrors of its
structs have the C layout, and argument checks that need no GPU behave."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sw_elliptic.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2103_16120_gb300 import build, _lib
    build.build()
    return _lib.load()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sw_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    from paper_2103_16120_gb300._lib import EXPORTS
    assert sorted(EXPORTS) == _declared_functions()


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    syms = set(re.findall(r"\bT (sw_[a-z_]+)\b", out))
    missing = [f for f in _declared_functions() if f not in syms]
    assert not missing, missing
    for f in _declared_functions():
        assert hasattr(lib, f)


def test_struct_layout_matches_c(tmp_path):
    from paper_2103_16120_gb300._lib import SolveOpts, SolveStats
    prog = tmp_path / "layout.c"
    fields_o = [f for f, _ in SolveOpts._fields_]
    fields_s = [f for f, _ in SolveStats._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){",
             'printf("%zu %zu\\n", sizeof(sw_solve_opts), sizeof(sw_solve_stats));']
    lines += [f'printf("%zu\\n", offsetof(sw_solve_opts, {f}));' for f in fields_o]
    lines += [f'printf("%zu\\n", offsetof(sw_solve_stats, {f}));' for f in fields_s]
    lines += ['printf("%zu %zu %zu %zu\\n", sizeof(sw_swe_params), offsetof(sw_swe_params, dt), '
              'offsetof(sw_swe_params, gravity), offsetof(sw_swe_params, omega));']
    lines += ['printf("%u\\n", (unsigned)SW_NOALLOC_SCRATCH_BYTES);', "return 0;}"]
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", str(prog), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals[0] == C.sizeof(SolveOpts) and vals[1] == C.sizeof(SolveStats)
    from paper_2103_16120_gb300._lib import SW_NOALLOC_SCRATCH_BYTES
    assert vals[-1] == SW_NOALLOC_SCRATCH_BYTES
    from paper_2103_16120_gb300._lib import SweParams
    assert vals[-5:-1] == [C.sizeof(SweParams)] + [getattr(SweParams, f).offset for f, _ in SweParams._fields_]
    offs = vals[2:-5]
    assert offs[: len(fields_o)] == [getattr(SolveOpts, f).offset for f in fields_o]
    assert offs[len(fields_o):] == [getattr(SolveStats, f).offset for f in fields_s]


def test_defaults_and_argument_checks_without_gpu(lib):
    from paper_2103_16120_gb300._lib import SolveOpts, SW_ERR_INVALID_ARG
    o = SolveOpts()
    lib.sw_solve_opts_default(C.byref(o))
    assert (o.k, o.tol, o.pc, o.n_richardson, o.prec, o.pole_band_rows) == (4, 1e-8, 3, 2, 0, -1)
    h = C.c_void_p()
    # odd nx, too small ny, bad radius: rejected before any CUDA call
    assert lib.sw_grid_create(7, 4, 1.0, C.byref(h)) == SW_ERR_INVALID_ARG
    assert b"nx" in lib.sw_last_error()
    assert lib.sw_grid_create(8, 1, 1.0, C.byref(h)) == SW_ERR_INVALID_ARG
    assert lib.sw_grid_create(8, 4, -1.0, C.byref(h)) == SW_ERR_INVALID_ARG
    assert lib.sw_grid_create(8192, 4, 1.0, C.byref(h)) == SW_ERR_INVALID_ARG
    assert lib.sw_gcr_solve(None, C.byref(o), None, None, None, None) == SW_ERR_INVALID_ARG
    assert lib.sw_ensemble_solve(1, None, C.byref(o), None, None, None, None) == SW_ERR_INVALID_ARG
    assert lib.sw_gcr_solve_noalloc(None, C.byref(o), None, None, None, None) == SW_ERR_INVALID_ARG
    from paper_2103_16120_gb300._lib import SweParams
    p = SweParams(600.0, 9.8, 7.292e-5)
    assert lib.sw_swe_create(None, C.byref(p), C.byref(h)) == SW_ERR_INVALID_ARG
    assert lib.sw_swe_create(None, None, None) == SW_ERR_INVALID_ARG
    assert lib.sw_swe_step(None, C.byref(o), 1, None, None) == SW_ERR_INVALID_ARG
    assert lib.sw_swe_set_state(None, None, None, None, None, None, None, None, None) == SW_ERR_INVALID_ARG
    assert lib.sw_swe_destroy(None) == 0


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import importlib
    from paper_2103_16120_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.load()
    importlib.reload(_lib)
