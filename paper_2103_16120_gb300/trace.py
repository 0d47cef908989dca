"""Device time line of the persistent solver (performance work).

The traced build of the library (``build.build(trace=True)``, compiled with
-DSW_PHASE_TRACE; same results) lets thread 0 of one chosen block record a
(globaltimer, tag) pair at fixed points of every phase.  ``timeline`` runs one
solve of a seeded synthetic problem with that build and returns the mean time
between consecutive tags, per tag pair.

Tags: 10 + phase at the start of a phase (phases: 0 true residual, 1 update,
2 Richardson stage, 3 L(e)), 30 after the row work, 31 after the block sums,
32 after the member barrier, 33 after the member sums, 35 after the L(e)
scalars, 36 after the state transition, 34 after the block has synchronised;
inside the rows 101/102 (L(e): staging, stencil), 201 (update
loop), 301/302/303 (stage: staging, stencil, zonal solve), 401/402 (first
stage: zonal solve, store); with one warp per row (warp 0 of the block) 111
(after L(e) and its inner products), 211/212/213 (first stage: before the
zonal solve, after it, after the store), 311/312/313 (stage: after the
stencil, the zonal solve, the store).

    python -m paper_2103_16120_gb300.trace NX NY PREC [BLOCK [ROW_MODE]]
"""
from __future__ import annotations

import collections
import ctypes as C
import json
import sys

import numpy as np


def timeline(nx: int, ny: int, prec: int, block: int = 0, seed: int = 1000, tol: float = 1e-8,
             row_mode: int = 0) -> dict:
    import torch

    from . import _lib as L
    from . import build as B
    if L._lib is not None:
        raise RuntimeError("timeline needs a process that has not loaded the library yet")
    L.LIB_PATH = B.build(trace=True)
    import paper_2103_16120_gb300 as sw
    import synth

    lib = L.load()
    lib.sw_trace_configure.argtypes = [C.c_void_p, C.c_int, C.c_int]
    P = synth.problem(nx, ny, seed)
    g = sw.sw_grid_create(nx, ny)
    sw.sw_elliptic_set_coeffs(g, *[torch.as_tensor(P[k], device="cuda") for k in sw.COEFF_KEYS])
    R = torch.as_tensor(P["R"], device="cuda")
    o = sw.sw_solve_opts_default(prec=prec, tol=tol, max_iters=5000, row_mode=row_mode)
    ms = []
    for _ in range(3):
        phi = torch.zeros_like(R)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        st = sw.sw_gcr_solve(g, o, R, phi)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    cap = 60000
    buf = torch.zeros(2 * cap, dtype=torch.int64, device="cuda")
    lib.sw_trace_configure(C.c_void_p(buf.data_ptr()), cap, block)
    phi = torch.zeros_like(R)
    st = sw.sw_gcr_solve(g, o, R, phi)
    torch.cuda.synchronize()
    lib.sw_trace_configure(C.c_void_p(0), 0, 0)
    t = buf.view(-1, 2).cpu().numpy()
    t = t[: int((t[:, 0] > 0).sum())]
    gaps = collections.defaultdict(list)
    for x, y in zip(t[:-1], t[1:]):
        gaps[(int(x[1]), int(y[1]))].append(int(y[0] - x[0]))
    return {"nx": nx, "ny": ny, "prec": prec, "block": block, "iterations": st.iterations,
            "ms": round(min(ms), 4), "us_per_iteration": round(1e3 * min(ms) / max(st.iterations, 1), 2),
            "ns": {f"{a}->{b}": [len(v), round(float(np.mean(v)))] for (a, b), v in sorted(gaps.items())
                   if len(v) > 2}}


if __name__ == "__main__":
    args = [int(a) for a in sys.argv[1:]]
    if len(args) < 3:
        sys.exit(__doc__)
    print(json.dumps(timeline(*args[:4], row_mode=args[4] if len(args) > 4 else 0)))
