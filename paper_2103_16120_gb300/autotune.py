"""Launch-shape autotuner for ensemble solves.

The tile of the solver kernel is one latitude row per thread block.  Its
width -- the threads that share a row, `threads_per_row` -- trades the
length of each thread's register chunk in the zonal scans against block-level
synchronisation and residency.  tune_ensemble times the candidate widths on
the caller's own ensemble (each candidate solved `reps` times from the same
first guesses, restored between runs) and keeps the fastest per ensemble
signature.  The timings use CUDA events on the current stream; every solve
runs in the library's kernels.
"""
from __future__ import annotations

from . import SW_OK, SolveOpts, sw_ensemble_solve

_CACHE: dict = {}


def _copy(opts: SolveOpts) -> SolveOpts:
    return SolveOpts.from_buffer_copy(opts)


def signature(grids, opts: SolveOpts) -> tuple:
    return (tuple((g.nx, g.ny) for g in grids), opts.prec, opts.k, opts.pc, opts.n_richardson)


def tune_ensemble(grids, opts: SolveOpts, Rs, phis, candidates=(64, 128, 256), reps: int = 2):
    """Returns (best opts, {threads_per_row: ms per ensemble}).  phis keep the
    caller's first guesses on return."""
    import torch
    key = signature(grids, opts)
    if key in _CACHE:
        best, table = _CACHE[key]
        o = _copy(opts)
        o.threads_per_row = best
        return o, table
    saved = [p.clone() for p in phis]
    stream = torch.cuda.current_stream()
    table = {}
    for tpr in candidates:
        o = _copy(opts)
        o.threads_per_row = tpr
        try:
            for p, s in zip(phis, saved):
                p.copy_(s)
            sw_ensemble_solve(grids, o, Rs, phis)                  # warm-up
            ms = 0.0
            for _ in range(reps):
                for p, s in zip(phis, saved):
                    p.copy_(s)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sts = sw_ensemble_solve(grids, o, Rs, phis)
                b.record(stream)
                torch.cuda.synchronize()
                if any(s.status != SW_OK for s in sts):
                    raise RuntimeError("candidate did not converge")
                ms += a.elapsed_time(b) / reps
            table[tpr] = ms
        except Exception:
            table[tpr] = float("inf")
    for p, s in zip(phis, saved):
        p.copy_(s)
    best = min(table, key=table.get)
    _CACHE[key] = (best, table)
    o = _copy(opts)
    o.threads_per_row = best
    return o, table
