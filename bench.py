"""Benchmark: elliptic solves/s to a 1e-8 relative residual on one GB300.

Default workload (one "step" = one elliptic solve of the sequence): a
sequence of 100 solves on a 2048 x 1024 lon/lat grid (about 2.1 M unknowns)
whose coefficients evolve smoothly between solves (seeded synthetic
shallow-water states, dt = 600 s), each warm-started from the previous
solution.  Each step runs the whole hot path through the C ABI:
sw_elliptic_set_coeffs (face coefficients, automatic eta, factorised zonal
operators) and the solve (GCR(4) with the semi-implicit Richardson
preconditioner, true residual <= 1e-8 ||R||), enqueued with
sw_ensemble_solve_async so that the host prepares the next step while the
GPU solves; every step's stats go to device memory and are checked after the
timed region.  The headline `value` is the mixed-precision solver (FP16
preconditioner storage with per-row scaling, FP32 operator and recursive
residual, FP64 inner products, solution and true residual); the plain FP64
GPU GCR is timed the same way and reported beside it, and so is the mixed
solver with the learned preconditioner (a network trained in the same run on
256 x 128 solver-generated triples and applied at 2048 x 1024 without
retraining).  The solution error of each arm is measured against the FP64
CPU oracle on the sequence's first problem.

The coefficient sets and right-hand sides of the timed steps (134 MB each)
are resident in HBM before timing; every set is larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload seq2048|seq512|learned256|ensemble64|swe512|oracle]

The other workloads measure the remaining configurations on one GPU, one
JSON line each:
  seq512      the same sequence measurement on a 512 x 256 grid (200 solves)
  learned256  the learned preconditioner at 256 x 128: GPU training on solver
              generated triples (tensor-core throughput against the BF16
              peak), then flexible-GCR solves against option 3 at 256 x 128
              and, without retraining, at 1024 x 512
  ensemble64  64 independent members (32 at 128x64, 24 at 256x128, 8 at
              512x256) in one persistent launch, against the same members
              solved one launch each
  swe512      the semi-implicit shallow-water model around the solver
              (Eqs. 1-10) at 512 x 256, dt = 200 s: model steps/s, two
              solves per step, mixed against FP64
  oracle      the CPU FP64 oracle on the host alone: seconds per solve of
              the workloads above, one thread and all host threads
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "elliptic solves/s at 1e-8 rel. residual: mixed+learned vs FP64 GCR, same GB300"
NX, NY, NSEQ, SEED, TOL, K_GCR = 512, 256, 200, 1000, 1e-8, 4
KEYS = ("A11", "A12", "A21", "A22", "B1", "B2", "C")

# the solve sequences: grid, length, seed of the seeded synthetic states
SEQS = {
    "seq2048": {"nx": 2048, "ny": 1024, "nseq": 100, "seed": 4000,
                "label": "sequence of 100 solves, 2048x1024 lon/lat grid, evolving coefficients, warm start"},
    "seq512": {"nx": 512, "ny": 256, "nseq": 200, "seed": 1000,
               "label": "sequence of 200 solves, 512x256 lon/lat grid, evolving coefficients, warm start"},
}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum, ncu) of the
# mixed-precision solver kernel per launch (seq512) or per GCR iteration
# (seq2048, scaled by the launch's iterations); None until captured for the
# current kernel
TRAFFIC = {"seq512": None, "seq2048_per_iteration": 70.40e9 / 275}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time: replicas are timed as one job."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_sequence(n: int, wl: str = "seq512"):
    q = SEQS[wl]
    return [synth.sequence_problem(q["nx"], q["ny"], q["seed"], t) for t in range(min(n, q["nseq"]))]


# ---------------------------------------------------------------------------
# CPU oracle leg (reported baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_solves(seq, budget_s: float, max_solves: int):
    import oracle as O
    ny, nx = seq[0]["C"].shape
    phi = np.zeros((ny, nx))
    t0 = time.perf_counter()
    n = 0
    its = []
    while n < max_solves:
        P = seq[n % len(seq)]
        phi, st = O.Problem(P).gcr(P["R"], O.Opts(k=K_GCR, tol=TOL, max_iters=4000), phi0=phi)
        its.append(st["iterations"])
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return n, dt, its


def oracle_reference_solve(P, tol: float = 1e-10):
    """The FP64 oracle's solve of one problem from a zero first guess, to tol.
    Returns the solution, the wall time, the iterations it took and the
    iteration at which its residual first met the benchmark tolerance."""
    import oracle as O
    t0 = time.perf_counter()
    phi, st, hist, _ = O.Problem(P).gcr(P["R"], O.Opts(k=K_GCR, tol=tol, max_iters=6000), want_history=True)
    dt = time.perf_counter() - t0
    at = np.nonzero(hist <= TOL)[0]
    its_tol = int(at[0]) if at.size else int(st["iterations"])
    return phi, dt, int(st["iterations"]), its_tol


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the host cores, on the same
    workload, metric and unit as the GPU arm.  seq512: each step is one
    warm-started oracle solve of the sequence.  seq2048: one oracle solve takes
    tens of seconds, so each step is a bounded sample of 16 GCR iterations of
    the sequence's next problem (warm-started from the previous step), and the
    time per iteration is scaled to solves/s by the iterations the oracle
    needs for the sequence's first problem (measured once, untimed).  Each
    sample also pays a solve's set-up (initial residual and preconditioner,
    final true residual, about 1.5 iterations of work), so the estimate
    over-states the oracle's time per solve by a few per cent."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    import oracle.oracle as orc
    orc.build()
    cores = cpu_cores()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    wl = args.workload if args.workload in SEQS else "seq2048"
    q = SEQS[wl]
    seq = make_sequence(args.steps + args.warmup + 1, wl)
    extra = {}
    if wl == "seq512":
        oracle_solves(seq, 1e9, args.warmup)   # warm-up solves (untimed)
        n, dt, its = oracle_solves(seq, 1e9, args.steps)
        v = n / dt
        ms = 1e3 * dt / n
        sample = f"{n} FP64 oracle solves of the 512x256 sequence (warm start), {cores} host threads"
        extra["mean_iterations"] = float(np.mean(its))
    else:
        _, _, its_full, its_tol = oracle_reference_solve(seq[0], tol=TOL)
        per = 16
        phi = np.zeros((q["ny"], q["nx"]))

        def sample_step(t):
            nonlocal phi
            P = seq[t % len(seq)]
            phi, st = O.Problem(P).gcr(P["R"], O.Opts(k=K_GCR, tol=0.0, max_iters=per), phi0=phi)

        for t in range(args.warmup):
            sample_step(t)
        t0 = time.perf_counter()
        for t in range(args.warmup, args.warmup + args.steps):
            sample_step(t)
        dt = time.perf_counter() - t0
        s_per_it = dt / (args.steps * per)
        v = 1.0 / (s_per_it * its_tol)
        ms = 1e3 / v
        sample = (f"{args.steps} steps of {per} FP64 oracle GCR iterations each on the 2048x1024 sequence "
                  f"(warm start), scaled by the {its_tol} iterations the oracle takes to 1e-8 on the first "
                  f"problem; {cores} host threads")
        extra["oracle_iterations_per_solve"] = its_tol
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": q["label"], "nx": q["nx"], "ny": q["ny"], "tol": TOL, "k": K_GCR,
                   "preconditioner": "semi-implicit Richardson, 2 iterations", "oracle": "CPU FP64"},
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        **extra,
    }), flush=True)


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during timing."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = os.path.join("/tmp", f"sw_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.out, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.out):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def algorithmic_bytes_per_point(prec_mixed: bool, its: float, stages: int = 2, k: int = K_GCR):
    """Minimum traffic of one GCR iteration per grid point with every listed
    phase fused (halo re-reads not counted), and of set-up + initial residual.

    FP64: beta-step (Phi rw 16, r rw 16, p 8, Lp 8) + sweep 1 (3 factors 24, q 8)
          + sweep 2 (q 8, r 8, 6 coefficients 48, 3 factors 24, e 8)
          + L(e) (e 8, 7 coefficients 56, Le 8, Lp_l 8 (nu+1))
          + update (e 8, Le 8, p_l and Lp_l 16 (nu+1), r 8, p and Lp 16)
    mixed: the same fields with r, p, Lp, Le, coefficients, factors in 4 bytes
           and q, e in 2 bytes; Phi stays FP64.
    (nu+1) averages (k+1)/2."""
    nu1 = (k + 1) / 2.0
    if not prec_mixed:
        beta = 16 + 16 + 8 + 8 + 24 + 8
        sweep2 = (8 + 8 + 48 + 24 + 8) * (stages - 1)
        le = 8 + 56 + 8 + 8 * nu1
        upd = 8 + 8 + 16 * nu1 + 8 + 16
    else:
        beta = 16 + 8 + 4 + 4 + 12 + 2
        sweep2 = (2 + 4 + 24 + 12 + 2) * (stages - 1)
        le = 2 + 28 + 4 + 4 * nu1
        upd = 2 + 4 + 8 * nu1 + 4 + 8
    per_it = beta + sweep2 + le + upd
    # set-up: read 7 FP64 cells, write FP64 + FP32 faces, diag, factors (FP64 + FP32)
    setup = 7 * 8 + 8 * 8 + 8 * 4 + 3 * 8 + 3 * 4 + 3 * 8
    # initial and final true residual: Phi 8, R 8, 7 FP64 coefficients 56, r write
    true_res = 2 * (8 + 8 + 56 + (4 if prec_mixed else 8))
    return per_it * its + setup + true_res


def learned_arm(sw, torch, dev, P, oracle_phi, n_states: int = 100, per_state: int = 40, epochs: int = 4):
    """The learned preconditioner beside the headline: a network trained in
    this run on n_states x per_state triples (R, L^-1 R) at 256 x 128 that the
    library's FP64 solver generates, then used without retraining in the mixed
    flexible GCR on problem P (zero first guess), against option 3 on the same
    problem.  Returns the measured solves, iterations and errors."""
    from paper_2103_16120_gb300 import learned
    t0 = time.perf_counter()
    probs = [synth.problem(256, 128, 3_000_000 + s) for s in range(n_states)]
    rhs = np.stack([synth.random_rhs(256, 128, 3_000_000 + s, per_state) for s in range(n_states)])
    m = sw.Model()
    sw.sw_model_set_params(m, learned.init_params(1))
    x0, tg = learned.make_dataset(m, probs, rhs)
    B = 32
    steps = max(1, epochs * x0.shape[0] // B)
    losses = learned.train(m, x0, tg, steps=steps, batch=B, lr=2e-3, seed=2)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del x0, tg
    ny, nx = P["C"].shape
    g = _grid(sw, torch, P, dev)
    R = torch.as_tensor(P["R"], device=dev)
    out = {"training": {"triples": n_states * per_state, "grid": "256x128", "epochs": epochs, "batch": B,
                        "steps": steps, "final_loss": losses[-1][1] if losses else None,
                        "data_and_training_s": t_train}}
    for tag, kw in (("option3", {}), ("learned", {"pc": sw.SW_PC_LEARNED, "model": m})):
        o = sw.sw_solve_opts_default(k=K_GCR, tol=TOL, prec=sw.SW_PREC_MIXED_FP16, max_iters=6000, **kw)
        phi = torch.zeros_like(R)
        st = sw.sw_gcr_solve(g, o, R, phi)         # first call: buffers and network set-up
        stream = torch.cuda.current_stream()
        phi.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = sw.sw_gcr_solve(g, o, R, phi)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        x = phi.cpu().numpy()
        out[tag] = {"ms_per_solve": ms, "solves_per_s": 1e3 / ms, "iterations": st.iterations,
                    "fallbacks": st.fallbacks, "status": int(st.status),
                    "true_rel_residual": st.true_rel_residual,
                    "solution_rel_error_vs_fp64_oracle": float(np.linalg.norm(x - oracle_phi) / np.linalg.norm(oracle_phi))}
    return out


def run_gpu(args):
    import torch
    import paper_2103_16120_gb300 as sw
    from paper_2103_16120_gb300 import build as swb

    wl = args.workload
    q = SEQS[wl]
    nx, ny, nseq = q["nx"], q["ny"], q["nseq"]
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    swb.build()
    dev = torch.device("cuda", local)

    # --- inputs resident in HBM -------------------------------------------
    # the sets the run visits (the sequence wraps after nseq solves)
    nsets = min(nseq, args.warmup + args.steps) if wl == "seq2048" else nseq
    seq = make_sequence(nsets, wl)
    coeffs = [[torch.as_tensor(P[k], device=dev) for k in KEYS] for P in seq]
    Rs = [torch.as_tensor(P["R"], device=dev) for P in seq]
    set_bytes = 8 * nx * ny * 8
    g = sw.sw_grid_create(nx, ny)
    stream = torch.cuda.current_stream()

    stat_bytes = sw.stats_buffer(1).numel()

    def run_steps(opts, phi, start, count, sbuf):
        # each step: the coefficients of the step, then the solve, enqueued
        # without a host synchronisation (stats of step i to sbuf slot i)
        for i, s_ in enumerate(range(start, start + count)):
            t = s_ % nsets
            sw.sw_elliptic_set_coeffs(g, *coeffs[t])
            sw.sw_ensemble_solve_async([g], opts, [Rs[t]], [phi], sbuf[i * stat_bytes:(i + 1) * stat_bytes])

    def checked(sbuf, count):
        sts = sw.stats_from_device(sbuf, count)
        for i, st in enumerate(sts):
            if st.status != sw.SW_OK:
                raise RuntimeError(f"solve {i} failed: {st.as_dict()}")
        return sts

    def timed(opts, K, W, clk=None):
        phi = torch.zeros((ny, nx), dtype=torch.float64, device=dev)
        wbuf, sbuf = sw.stats_buffer(max(W, 1)), sw.stats_buffer(K)
        wopts = sw.SolveOpts.from_buffer_copy(opts)
        wopts.split_r0 = 0          # the warm-up steps come before the first refresh
        run_steps(wopts, phi, 0, W, wbuf)
        torch.cuda.synchronize()
        checked(wbuf, W)
        if opts.split_r0:
            # Phi_hat of Eq. 14 refreshed once, from the last warm-up solution
            sw.sw_split_refresh(g, phi)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if clk is not None:
            clk.start()
        ev0.record(stream)
        run_steps(opts, phi, W, K, sbuf)
        ev1.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop() if clk is not None else None
        if world > 1:
            torch.distributed.barrier()
        sts = checked(sbuf, K)
        ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
        return ms, sts, clocks

    maxit = 6000
    mixed = sw.sw_solve_opts_default(k=K_GCR, tol=TOL, prec=sw.SW_PREC_MIXED_FP16, max_iters=maxit,
                                     pole_band_rows=args.pole_band, ru_every=args.ru_every,
                                     split_r0=int(args.split_r0))
    fp64 = sw.sw_solve_opts_default(k=K_GCR, tol=TOL, prec=sw.SW_PREC_FP64, max_iters=maxit)

    # FP64 reference path first (same steps), then the mixed path with clocks
    ms64, st64, _ = timed(fp64, args.steps, args.warmup)
    msm, stm, clocks = timed(mixed, args.steps, args.warmup, ClockSampler(local))

    # --- kernel-only timing of the solver kernel (dominant kernel) ---------
    # events around sw_gcr_solve alone: the persistent GCR kernel plus one
    # descriptor kernel and two tiny state copies
    def solver_only(opts, K):
        phi = torch.zeros((ny, nx), dtype=torch.float64, device=dev)
        tot, its = 0.0, 0
        for s_ in range(K):
            t = s_ % nsets
            sw.sw_elliptic_set_coeffs(g, *coeffs[t])
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = sw.sw_gcr_solve(g, opts, Rs[t], phi)
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
            its += st.iterations
        return tot / K, its / K

    kms, kits = solver_only(mixed, min(args.steps, 50 if wl == "seq512" else 8))

    # --- end to end through host buffers ----------------------------------
    # every step copies its coefficients and R from pinned host memory and
    # reads its solution back; the copies of step s + 1 run on a copy stream
    # into the second of two device buffer sets while step s solves
    n_host = min(nsets, 50 if wl == "seq512" else 10)   # one host set per timed step: no wrap of the sequence
    hcoef = [[torch.as_tensor(P[k]).pin_memory() for k in KEYS] for P in seq[:n_host]]
    hR = [torch.as_tensor(P["R"]).pin_memory() for P in seq[:n_host]]
    hphi = torch.zeros((ny, nx), dtype=torch.float64).pin_memory()
    dco = [[torch.empty((ny, nx), dtype=torch.float64, device=dev) for _ in KEYS] for _ in range(2)]
    dR = [torch.empty((ny, nx), dtype=torch.float64, device=dev) for _ in range(2)]
    dphi = torch.zeros((ny, nx), dtype=torch.float64, device=dev)
    n_e2e = min(args.steps, 50 if wl == "seq512" else 10)
    ebuf = sw.stats_buffer(max(n_e2e, 3))
    cstream = torch.cuda.Stream(device=dev)
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    free = [torch.cuda.Event(), torch.cuda.Event()]
    # the solution read back through a device copy, also on the copy stream
    dout = [torch.empty((ny, nx), dtype=torch.float64, device=dev) for _ in range(2)]
    solved = [torch.cuda.Event(), torch.cuda.Event()]
    read = [torch.cuda.Event(), torch.cuda.Event()]

    def h2d(s_):
        b, t = s_ % 2, s_ % len(hR)
        with torch.cuda.stream(cstream):
            cstream.wait_event(free[b])          # the solve that last read buffer set b is done
            for d, h in zip(dco[b], hcoef[t]):
                d.copy_(h, non_blocking=True)
            dR[b].copy_(hR[t], non_blocking=True)
            ready[b].record(cstream)

    def e2e_steps(n):
        for b in range(2):
            free[b].record(stream)
            read[b].record(stream)
        h2d(0)
        for s_ in range(n):
            b = s_ % 2
            if s_ + 1 < n:
                h2d(s_ + 1)
            stream.wait_event(ready[b])
            sw.sw_elliptic_set_coeffs(g, *dco[b])
            sw.sw_ensemble_solve_async([g], mixed, [dR[b]], [dphi], ebuf[s_ * stat_bytes:(s_ + 1) * stat_bytes])
            free[b].record(stream)
            stream.wait_event(read[b])              # the read-back that last used dout[b] is done
            dout[b].copy_(dphi)
            solved[b].record(stream)
            with torch.cuda.stream(cstream):
                cstream.wait_event(solved[b])
                hphi.copy_(dout[b], non_blocking=True)
                read[b].record(cstream)
        torch.cuda.synchronize()
        checked(ebuf, n)

    e2e_steps(min(args.warmup, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps(n_e2e)
    e2e_dt = time.perf_counter() - t0
    h2d = set_bytes
    d2h = nx * ny * 8

    # --- solution error against the FP64 oracle, CPU baseline, learned arm --
    # every arm solves the sequence's first problem from a zero first guess;
    # the oracle solves it to 1e-10
    err = err64 = None
    cpu = None
    learned_out = None
    if rank == 0:
        import oracle.oracle as orc
        orc.build()
        cores = cpu_cores()
        os.environ.setdefault("OMP_NUM_THREADS", str(cores))
        P0 = seq[0]
        ref, t_or, its_or, its_or_tol = oracle_reference_solve(P0)
        sw.sw_elliptic_set_coeffs(g, *coeffs[0])
        for tag, o in (("mixed", mixed), ("fp64", fp64)):
            phi0 = torch.zeros((ny, nx), dtype=torch.float64, device=dev)
            st = sw.sw_gcr_solve(g, o, Rs[0], phi0)
            if st.status != sw.SW_OK:
                raise RuntimeError(f"{tag} solve of the first problem failed: {st.as_dict()}")
            e_ = float(np.linalg.norm(phi0.cpu().numpy() - ref) / np.linalg.norm(ref))
            if tag == "mixed":
                err = e_
            else:
                err64 = e_
        if wl == "seq512":
            # bounded CPU-oracle sample on the host cores
            n, dt, its = oracle_solves(seq, 15.0, 200)
            cpu = {"value": n / dt, "unit": "solves/s", "cores": cores, "kind": "oracle",
                   "sample": f"first {n} solves of the same 512x256 sequence, FP64 oracle, warm start, "
                             f"OpenMP over rows ({cores} threads), {dt:.1f} s"}
        else:
            v_or = its_or / (t_or * its_or_tol)
            cpu = {"value": v_or, "unit": "solves/s", "cores": cores, "kind": "oracle",
                   "sample": f"one FP64 oracle solve of the sequence's first 2048x1024 problem from zero, "
                             f"{its_or} iterations to 1e-10 in {t_or:.1f} s, scaled to the {its_or_tol} "
                             f"iterations that reach 1e-8; OpenMP over rows ({cores} threads)"}
            if not args.no_learned:
                learned_out = learned_arm(sw, torch, dev, P0, ref)
                m3, ml = learned_out["option3"], learned_out["learned"]
                learned_out["gain_vs_option3"] = m3["ms_per_solve"] / ml["ms_per_solve"]
                learned_out["shipped"] = "learned" if ml["ms_per_solve"] < m3["ms_per_solve"] else "option3"
                if learned_out["shipped"] == "option3":
                    learned_out["reason"] = (
                        "the learned directions cost more than they save: each network turn ends the persistent "
                        "launch and round-trips through the host, and the network's +-15-point receptive field "
                        "cannot represent the coupling around whole latitude circles that option 3 solves "
                        "exactly; the headline is the mixed-precision solver with option 3")

    its_m = float(np.mean([s_.iterations for s_ in stm]))
    its_64 = float(np.mean([s_.iterations for s_ in st64]))
    value = world * args.steps / (msm / 1e3)
    v64 = world * args.steps / (ms64 / 1e3)
    bpp = algorithmic_bytes_per_point(True, kits)
    achieved = bpp * nx * ny / (kms / 1e3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    if wl == "seq512":
        traffic = TRAFFIC["seq512"]
        note = ("algorithmic bytes of one solve / solver time; working set is L2-resident "
                "and the solve is grid-barrier-latency bound at this size")
    else:
        tpi = TRAFFIC["seq2048_per_iteration"]
        traffic = tpi * kits if tpi else None
        note = ("algorithmic bytes of one solve / solver time (persistent kernel, mean iterations of the "
                "measured launches); traffic: ncu DRAM bytes per iteration of one launch times those iterations")
    launches_per_step = 4   # k_faces, k_factor<float>, k_init_one, k_gcr
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": msm / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f16 storage, f64 reductions)",
            "data": "synthetic",
            "config": {"workload": q["label"], "nx": nx, "ny": ny, "tol": TOL, "k": K_GCR,
                       "preconditioner": "semi-implicit Richardson, 2 iterations (option 3); learned arm beside",
                       "precision": "mixed-fp16",
                       "pole_band_rows": "automatic (the paper's angular width)" if args.pole_band < 0 else args.pole_band,
                       "ru_every": args.ru_every,
                       "initial_residual": "FP32, split fluid thickness (Eq. 14), refreshed before the timed steps"
                                           if args.split_r0 else "FP64",
                       "l2": f"inputs larger than L2 ({nsets} resident coefficient sets, {nsets * set_bytes / 1e9:.1f} GB)",
                       "parallelism": f"replicas x{world}"},
            "fp64_gcr": {"value": v64, "unit": "solves/s", "ms_per_step": ms64 / args.steps,
                         "mean_iterations": its_64, "solution_rel_error_vs_fp64_oracle": err64},
            "speedup_vs_fp64": value / v64,
            "mean_iterations": its_m,
            "solution_rel_error_vs_fp64_oracle": err,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": ("k_gcr<PolF16> (persistent GCR, one warp per row, specialised for rows of 2048 points)"
                                    if wl == "seq2048" else "k_gcr<PolF16> (persistent GCR)"),
                         "kernel_ms_per_launch": kms, "kernel_mean_iterations": kits,
                         "algorithmic_bytes_per_point": bpp, "note": note,
                         "peak_source": "measured hbm_gbs (of measured)" if peaks else "fallback 6800 GB/s"},
            "cpu_baseline": cpu,
            "e2e": {"value": world * n_e2e / e2e_dt, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
        }
        if learned_out is not None:
            line["learned"] = learned_out
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# further workloads (one GPU)
# ---------------------------------------------------------------------------
def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _oracle_baseline(problems, budget_s: float, what: str):
    """The FP64 oracle on the host cores over a bounded sample of problems
    (zero first guess, tol 1e-8): member solves per second."""
    import oracle as O
    import oracle.oracle as orc
    orc.build()
    cores = cpu_cores()
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < budget_s and n < 100 * len(problems):
        P = problems[n % len(problems)]
        O.Problem(P).gcr(P["R"], O.Opts(k=K_GCR, tol=TOL, max_iters=4000))
        n += 1
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{what}: {n} solves (the {len(problems)} problems in turn) in {dt:.1f} s, "
                      f"OpenMP over rows ({cores} threads)"}


def _grid(sw, torch, P, dev):
    ny, nx = P["C"].shape
    g = sw.sw_grid_create(nx, ny)
    sw.sw_elliptic_set_coeffs(g, *[torch.as_tensor(P[k], device=dev) for k in KEYS])
    return g


# kernels of one learned solve: the solver's first launch and the graph's first
# test of the member's state, then per network turn the graph body's kernels
# (sum of squares and features of r, input packing, 6 convolutions, 2 poolings,
# 2 upsample + concatenations, output scaling, e stored in the member's format,
# the resumed solver, the state test)
LEARNED_LAUNCHES_PER_SOLVE, LEARNED_LAUNCHES_PER_TURN = 2, 17


def _time_solves(sw, torch, g, opts, Rs, reps, turns=None):
    """Mean solve time (CUDA events) and mean iterations over reps solves
    (network turns of each solve appended to `turns` when given)."""
    stream = torch.cuda.current_stream()
    tot, its, fb = 0.0, 0, 0
    for q in range(reps):
        R = Rs[q % len(Rs)]
        phi = torch.zeros_like(R)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = sw.sw_gcr_solve(g, opts, R, phi)
        b.record(stream)
        torch.cuda.synchronize()
        if st.status != sw.SW_OK:
            raise RuntimeError(f"solve failed: {st.as_dict()}")
        tot += a.elapsed_time(b)
        its += st.iterations
        fb += st.fallbacks
        if turns is not None:
            turns.append(st.network_turns)
    return tot / reps, its / reps, fb / reps


def run_learned(args):
    import torch
    import paper_2103_16120_gb300 as sw
    from paper_2103_16120_gb300 import build as swb, learned
    swb.build()
    dev = torch.device("cuda", 0)
    nx, ny = 256, 128
    n_states, per_state = max(1, args.samples // 40), 40
    t0 = time.perf_counter()
    probs = [synth.problem(nx, ny, 3_000_000 + s) for s in range(n_states)]
    rhs = np.stack([synth.random_rhs(nx, ny, 3_000_000 + s, per_state) for s in range(n_states)])
    m = sw.Model()
    sw.sw_model_set_params(m, learned.init_params(1))
    x0, tg = learned.make_dataset(m, probs, rhs)
    t_data = time.perf_counter() - t0
    # training throughput: K timed AdamW steps of batch 32 after W warm-up steps
    B = 32
    n = x0.shape[0]
    stream = torch.cuda.current_stream()
    learned.train(m, x0, tg, steps=args.warmup, batch=B, lr=1e-3)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(0)
    clk.start()
    a.record(stream)
    learned.train(m, x0, tg, steps=args.steps, batch=B, lr=1e-3, seed=1)
    b.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms_step = a.elapsed_time(b) / args.steps
    # then train to the end of the epochs asked for
    epochs_steps = max(0, args.epochs * n // B - args.steps - args.warmup)
    losses = learned.train(m, x0, tg, steps=epochs_steps, batch=B, lr=2e-3, seed=2) if epochs_steps else []
    flops = learned.train_flops_per_point() * nx * ny * B
    tflops = flops / (ms_step * 1e-3) / 1e12
    peak = _peaks().get("bf16_tflops", 1900.0)
    out = {}
    turns = {(gx, tag): [] for gx in (256, 1024) for tag in ("option3", "learned")}
    for (gx, gy) in ((256, 128), (1024, 512)):
        Ps = [synth.problem(gx, gy, 4_000_000 + s) for s in range(2)]
        res = {}
        for tag, kw in (("option3", {}), ("learned", {"pc": sw.SW_PC_LEARNED, "model": m})):
            o = sw.sw_solve_opts_default(k=K_GCR, tol=TOL, prec=sw.SW_PREC_MIXED_FP16, max_iters=2000, **kw)
            ms, its, fb = 0.0, 0.0, 0.0
            for P in Ps:
                g = _grid(sw, torch, P, dev)
                R = torch.as_tensor(P["R"], device=dev)
                _time_solves(sw, torch, g, o, [R], 1)
                a_, b_, c_ = _time_solves(sw, torch, g, o, [R], 3, turns[(gx, tag)])
                ms += a_ / len(Ps); its += b_ / len(Ps); fb += c_ / len(Ps)
            res[tag] = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "mean_iterations": its, "mean_fallbacks": fb,
                        "mean_network_turns": sum(turns[(gx, tag)]) / len(turns[(gx, tag)])}
        out[f"{gx}x{gy}"] = res
    head = out["256x128"]["learned"]
    print(json.dumps({
        "metric": METRIC, "value": head["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_solve"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 network (f32 accumulate), f32/f16 solver", "data": "synthetic",
        "config": {"workload": "learned preconditioner at 256x128, evaluated at 256x128 and 1024x512", "samples": n,
                   "epochs": args.epochs, "batch": B, "network": "3-level U-Net 32/64/64, 158369 parameters"},
        "solves": out,
        "training": {"ms_per_step": ms_step, "samples_per_s": B / (ms_step * 1e-3), "tflops": tflops,
                     "data_generation_s": t_data, "final_loss": losses[-1][1] if losses else None},
        "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                     "frac": tflops / peak, "traffic": None,
                     "kernel": "training step (tcgen05 forward and c4/c5 weight gradients, mma.sync input "
                               "gradients and the other weight gradients, BF16 operands, FP32 accumulation)",
                     "note": "algorithmic FLOPs of forward + input and weight gradients per step / step time",
                     "peak_source": "measured bf16_tflops (of measured)"},
        "cpu_baseline": _oracle_baseline([synth.problem(256, 128, 4_000_000 + s_) for s_ in range(2)], 10.0,
                                         "FP64 oracle option-3 solves of the 256x128 evaluation problems"),
        # the headline's timed solves (the learned ones at 256 x 128)
        "gpu_launches": sum(LEARNED_LAUNCHES_PER_SOLVE + LEARNED_LAUNCHES_PER_TURN * t for t in turns[(256, "learned")]),
        "clocks": clocks,
    }), flush=True)


def run_ensemble(args):
    import torch
    import paper_2103_16120_gb300 as sw
    from paper_2103_16120_gb300 import build as swb
    swb.build()
    dev = torch.device("cuda", 0)
    members = synth.ensemble_members()
    Ps = [synth.problem(nx, ny, seed) for nx, ny, seed in members]
    grids = [_grid(sw, torch, P, dev) for P in Ps]
    Rs = [torch.as_tensor(P["R"], device=dev) for P in Ps]
    phis = [torch.zeros_like(R) for R in Rs]
    o = sw.sw_solve_opts_default(k=K_GCR, tol=TOL, prec=sw.SW_PREC_MIXED_FP16, max_iters=2000)
    stream = torch.cuda.current_stream()

    def one(batched: bool):
        for p in phis:
            p.zero_()
        if batched:
            return sw.sw_ensemble_solve(grids, o, Rs, phis)
        return [sw.sw_gcr_solve(g, o, R, p) for g, R, p in zip(grids, Rs, phis)]

    from paper_2103_16120_gb300 import autotune
    o, table = autotune.tune_ensemble(grids, o, Rs, phis)
    res = {}
    for tag, batched in (("one_launch", True), ("launch_per_member", False)):
        for _ in range(args.warmup):
            one(batched)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            sts = one(batched)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        bad = [s.as_dict() for s in sts if s.status != sw.SW_OK]
        if bad:
            raise RuntimeError(f"ensemble member failed: {bad[0]}")
        res[tag] = {"ms_per_ensemble": ms, "member_solves_per_s": len(grids) / (ms * 1e-3),
                    "iterations": [s.iterations for s in sts]}
    # the same one-launch solve recorded once in a CUDA graph and replayed
    buf = sw.stats_buffer(len(grids))
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    cap.wait_stream(stream)
    with torch.cuda.stream(cap):
        with torch.cuda.graph(graph, stream=cap):
            for p in phis:
                p.zero_()
            sw.sw_ensemble_solve_async(grids, o, Rs, phis, buf)
    stream.wait_stream(cap)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(0)
    clk.start()
    a.record(stream)
    for _ in range(args.steps):
        graph.replay()
    b.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    gms = a.elapsed_time(b) / args.steps
    gst = sw.stats_from_device(buf, len(grids))
    if any(s_.status != sw.SW_OK for s_ in gst):
        raise RuntimeError("graph replay: a member failed")
    res["graph_replay"] = {"ms_per_ensemble": gms, "member_solves_per_s": len(grids) / (gms * 1e-3),
                           "iterations": [s_.iterations for s_ in gst]}
    head = res["graph_replay"] if gms < res["one_launch"]["ms_per_ensemble"] else res["one_launch"]
    pts_its = sum(nx * ny * it for (nx, ny, _), it in zip(members, head["iterations"]))
    bytes_ = algorithmic_bytes_per_point(True, 1) - algorithmic_bytes_per_point(True, 0)
    achieved = bytes_ * pts_its / (head["ms_per_ensemble"] * 1e-3) / 1e9
    peak = _peaks().get("hbm_gbs", 6800.0)
    print(json.dumps({
        "metric": METRIC, "value": head["member_solves_per_s"], "unit": "solves/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_ensemble"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f16 storage, f64 reductions)",
        "data": "synthetic",
        "config": {"workload": "ensemble of 64 members (32 at 128x64, 24 at 256x128, 8 at 512x256) in one persistent launch",
                   "members": "32 x 128x64, 24 x 256x128, 8 x 512x256", "tol": TOL, "precision": "mixed-fp16"},
        "launch_per_member": res["launch_per_member"], "one_launch": res["one_launch"],
        "graph_replay": res["graph_replay"],
        "autotune_ms_by_threads_per_row": table, "threads_per_row": o.threads_per_row,
        "speedup_vs_launch_per_member": res["launch_per_member"]["ms_per_ensemble"] / head["ms_per_ensemble"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "k_gcr<PolF16> (all members, one launch)",
                     "note": "algorithmic bytes (172 B per point per iteration) / ensemble time",
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
        "cpu_baseline": _oracle_baseline(Ps, 15.0, "FP64 oracle solves of the ensemble members one after another"),
        # per replay: the members' initial state (k_init_members) and the solve (k_gcr)
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
    }), flush=True)


# bytes per cell of one model step moved by the kernels around the solves
# (fields of 8 bytes unless noted): forcing 9 in / 7 out; transport 4 / 2;
# per pass (two passes): coefficients 10-11 / 11, face coefficients 7 / 8 plus
# 8 FP32 copies, FP32 zonal factors 2 / 3 FP32, L(Phi^n) 8 / 1, right-hand
# side 4 / 1; the first guess 2 / 1 and its copy 2; recovery 8 / 3
SWE_EXPLICIT_BYTES = 8 * (16 + 6 + (21 + 22) + 5 + 9 + 4) + 2 * (7 * 8 + 8 * 8 + 8 * 4) + 2 * (16 + 12) \
    + 2 * (8 + 56 + 8) + 2 * 40


def run_swe(args):
    """Semi-implicit shallow-water time stepping around the solve (Eqs. 1-10)
    at 512 x 256 with the paper's dt = 200 s: model steps/s, each step two
    solves (predictor and corrector), mixed FP16 against FP64."""
    import torch
    import paper_2103_16120_gb300 as sw
    from paper_2103_16120_gb300 import build as swb
    swb.build()
    dev = torch.device("cuda", 0)
    nx, ny = NX, NY
    dt = synth.paper_dt(ny)
    s0 = synth.perturbed_state(nx, ny, 5000, dt=dt, orography=500.0)
    fields = [s0.phi, s0.qx, s0.qy, s0.h0, s0.alpha, s0.qbar_x, s0.qbar_y]
    init = [torch.as_tensor(f, device=dev) for f in fields]
    g = sw.sw_grid_create(nx, ny)
    m = sw.sw_swe_create(g, dt)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # larger than the 129 MB L2
    K, W = args.steps, args.warmup
    out = {}
    clk = ClockSampler(0)
    for tag, prec in (("fp64", sw.SW_PREC_FP64), ("mixed", sw.SW_PREC_MIXED_FP16)):
        o = sw.sw_solve_opts_default(k=K_GCR, tol=TOL, prec=prec, max_iters=2000)
        # iterations and convergence from an identical run with the solves' stats
        sw.sw_swe_set_state(m, *init)
        stats = sw.sw_swe_step(m, o, W + K)
        bad = [x.as_dict() for x in stats if x.converged != 1]
        if bad:
            raise RuntimeError(f"{tag}: a solve did not converge: {bad[0]}")
        its = [x.iterations for x in stats[2 * W:]]
        # timed: L2 flushed before every step, events on the launching stream
        sw.sw_swe_set_state(m, *init)
        sw.sw_swe_step(m, o, W, want_stats=False)
        if tag == "mixed":
            clk.start()
        tot = 0.0
        for _ in range(K):
            flush.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sw.sw_swe_step(m, o, 1, want_stats=False)
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        if tag == "mixed":
            clocks = clk.stop()
        phi = torch.empty((ny, nx), dtype=torch.float64, device=dev)
        sw.sw_swe_get_state(m, phi)
        torch.cuda.synchronize()
        out[tag] = {"ms_per_step": tot / K, "steps_per_s": 1e3 * K / tot,
                    "solver_iterations_per_step": 2 * float(np.mean(its)) if its else 0.0,
                    "predictor_iterations": float(np.mean(its[0::2])), "corrector_iterations": float(np.mean(its[1::2])),
                    "phi": phi.cpu().numpy()}
    mixed, f64 = out["mixed"], out["fp64"]
    dphi64 = f64["phi"] - s0.phi
    err = float(np.max(np.abs(mixed["phi"] - f64["phi"])) / np.max(np.abs(dphi64)))
    cw = np.cos(synth.grid_coords(nx, ny)[1])[:, None]
    mass_drift = float(abs(np.sum(cw * mixed["phi"]) - np.sum(cw * s0.phi)) / np.sum(cw * s0.phi))
    # end to end through the public API: state in from pinned host memory, K
    # steps, state out to pinned host memory
    o = sw.sw_solve_opts_default(k=K_GCR, tol=TOL, prec=sw.SW_PREC_MIXED_FP16, max_iters=2000)
    hin = [torch.as_tensor(f).pin_memory() for f in fields]
    hout = [torch.empty((ny, nx), dtype=torch.float64).pin_memory() for _ in range(3)]
    din = [torch.empty((ny, nx), dtype=torch.float64, device=dev) for _ in fields]
    dout = [torch.empty((ny, nx), dtype=torch.float64, device=dev) for _ in range(3)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for d, h in zip(din, hin):
        d.copy_(h, non_blocking=True)
    sw.sw_swe_set_state(m, *din)
    sw.sw_swe_step(m, o, K, want_stats=False)
    sw.sw_swe_get_state(m, *dout)
    for d, h in zip(dout, hout):
        h.copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    # CPU oracle: the same model steps, bounded sample
    from oracle.swe import Stepper
    from oracle import Opts
    st = Stepper(nx, ny, dt, h0=s0.h0, alpha=s0.alpha, qbar_x=s0.qbar_x, qbar_y=s0.qbar_y)
    p, qx, qy, up, vp = s0.phi, s0.qx, s0.qy, None, None
    t0 = time.perf_counter()
    n_or = 0
    while n_or < 40 and time.perf_counter() - t0 < 12.0:
        p, qx, qy, up, vp, _ = st.step(p, qx, qy, up, vp, Opts(k=K_GCR, tol=TOL, max_iters=2000))
        n_or += 1
    or_s = time.perf_counter() - t0
    step_bytes = SWE_EXPLICIT_BYTES * nx * ny + algorithmic_bytes_per_point(
        True, mixed["solver_iterations_per_step"]) * nx * ny
    achieved = step_bytes / (mixed["ms_per_step"] * 1e-3) / 1e9
    peak = _peaks().get("hbm_gbs", 6800.0)
    print(json.dumps({
        "metric": "semi-implicit model steps/s (two elliptic solves per step, 1e-8 rel. residual)",
        "value": mixed["steps_per_s"], "unit": "steps/s", "n_gpus": 1, "steps": K, "warmup": W,
        "ms_per_step": mixed["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 model, f32 solver (f16 storage, f64 reductions)", "data": "synthetic",
        "config": {"workload": "semi-implicit shallow-water time stepping, 512x256, dt 200 s, perturbed balanced "
                               "flow over 500 m orography, polar absorber",
                   "nx": nx, "ny": ny, "dt_s": dt, "tol": TOL, "k": K_GCR,
                   "l2": "flushed (256 MB write) before every timed step"},
        "fp64_gcr": {k: v for k, v in f64.items() if k != "phi"},
        "mixed": {k: v for k, v in mixed.items() if k != "phi"},
        "speedup_vs_fp64": mixed["steps_per_s"] / f64["steps_per_s"],
        "phi_difference_mixed_vs_fp64_rel_to_fp64_change": err,
        "relative_mass_change": mass_drift,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "whole step (k_gcr dominant; see the launch list)",
                     "note": "algorithmic bytes of the step (stepper kernels + two solves) / step time; "
                             "the 37 MB state is latency-bound in the solves",
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
        "cpu_baseline": {"value": n_or / or_s, "unit": "steps/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": f"first {n_or} steps of the same run, FP64 oracle (two solves per step), "
                                   f"{or_s:.1f} s"},
        "e2e": {"value": K / e2e_s, "unit": "steps/s",
                "h2d_bytes_per_step": 7 * nx * ny * 8 // K, "d2h_bytes_per_step": 3 * nx * ny * 8 // K},
        "gpu_launches": 18 * K,
        "clocks": clocks,
    }), flush=True)


def run_oracle_timings(args):
    """CPU oracle timings of the benchmark's workloads, one host thread and all
    of them: the 128x64 single solve (20 solves, tol 1e-10), the first 10
    solves of the 512x256 sequence, 2 solves of the 2048x1024 sequence (warm
    start, tol 1e-8) and the 64 ensemble members one after another.  A
    reported baseline, not a target; no GPU is used."""
    import oracle as O
    import oracle.oracle as orc
    orc.build()
    cores = cpu_cores()
    cases = [
        ("128x64 single solve, tol 1e-10", [synth.problem(128, 64, 0)] * 20, False, 1e-10),
        ("512x256 sequence, first 10 solves", [synth.sequence_problem(NX, NY, SEED, t) for t in range(10)], True, TOL),
        ("2048x1024 sequence, 2 solves", [synth.sequence_problem(2048, 1024, 4000, t) for t in range(2)], True, TOL),
        ("ensemble members one after another",
         [synth.problem(nx, ny, seed) for nx, ny, seed in synth.ensemble_members()], False, TOL),
    ]
    rows = {}
    for label, probs, warm, tol in cases:
        rows[label] = {}
        for nth in (1, cores):
            orc.set_threads(nth)
            phi, its = None, []
            t0 = time.perf_counter()
            for P in probs:
                phi, st = O.Problem(P).gcr(P["R"], O.Opts(k=K_GCR, tol=tol, max_iters=5000),
                                           phi0=phi if warm else None)
                its.append(st["iterations"])
            dt = time.perf_counter() - t0
            rows[label][f"threads_{nth}"] = {"s_per_solve": dt / len(probs), "solves": len(probs),
                                             "mean_iterations": float(np.mean(its))}
    orc.set_threads(cores)
    print(json.dumps({"impl": "oracle", "metric": "CPU FP64 oracle seconds per solve", "unit": "s/solve",
                      "higher_is_better": False, "cores": cores, "data": "synthetic", "timings": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gcr", choices=["gcr", "reference"])
    ap.add_argument("--workload", default="seq2048",
                    choices=["seq2048", "seq512", "learned256", "ensemble64", "swe512", "oracle"])
    ap.add_argument("--no-learned", action="store_true", help="seq2048: leave the learned arm out")
    ap.add_argument("--pole-band", type=int, default=-1,
                    help="seq2048/seq512 mixed arm: FP32 rows at each pole (-1: the paper's angular width)")
    ap.add_argument("--split-r0", action="store_true",
                    help="seq2048/seq512 mixed arm: initial residual by the split form of Eq. 14")
    ap.add_argument("--ru-every", type=int, default=0,
                    help="seq2048/seq512 mixed arm: FP64 true residual every N iterations (0: at the exit test)")
    ap.add_argument("--samples", type=int, default=20000, help="learned256: training triples")
    ap.add_argument("--epochs", type=int, default=4, help="learned256: training epochs")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "learned256":
        run_learned(args)
    elif args.workload == "ensemble64":
        run_ensemble(args)
    elif args.workload == "swe512":
        run_swe(args)
    elif args.workload == "oracle":
        run_oracle_timings(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
