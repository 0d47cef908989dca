"""Training of the learned preconditioner on the GPU.

Orchestration only: the samples come from the library's own FP64 GCR solver,
and every step of the forward pass, backward pass and AdamW update runs in the
library's kernels (sw_model_train_step).  Host code only picks the
mini-batches.

A sample is a pair (R, Phi = L^-1 R) on a grid with seeded coefficients.  In
flexible GCR the network's directions e = s y / d alternate with those of the
paper's preconditioner, so its target is the solution itself:
y* = |diag L| Phi / rms(R), or with target="p3_error" the error of option 3,
|diag L| (Phi - P3(R)) / rms(R).  The inputs x0 = features(R) and the target
come from sw_model_features and sw_model_target.
"""
from __future__ import annotations

import math

import numpy as np

from . import (COEFF_KEYS, Model, SW_OK, SW_PC_SI_RICHARDSON, SW_PREC_FP64, sw_elliptic_set_coeffs,
               sw_gcr_solve, sw_grid_create, sw_model_features, sw_model_target, sw_model_train_step,
               sw_precond_apply, sw_solve_opts_default)


def make_dataset(model: Model, problems, rhs, tol: float = 1e-10, n_richardson: int = 2,
                 target: str = "solution"):
    """problems: list of coefficient dicts (numpy, [ny][nx]); rhs: array
    [n_problems, n_rhs, ny, nx] of right-hand sides.  Returns device tensors
    x0 [N, 4, ny, nx] and target [N, ny, nx] (FP32), N = n_problems * n_rhs."""
    import torch
    ny, nx = problems[0]["C"].shape
    n = len(problems) * rhs.shape[1]
    x0 = torch.empty((n, 4, ny, nx), dtype=torch.float32, device="cuda")
    tg = torch.empty((n, ny, nx), dtype=torch.float32, device="cuda")
    opts = sw_solve_opts_default(prec=SW_PREC_FP64, tol=tol, max_iters=5000)
    popts = sw_solve_opts_default(prec=SW_PREC_FP64, pc=SW_PC_SI_RICHARDSON, n_richardson=n_richardson)
    q = 0
    for p, P in enumerate(problems):
        g = sw_grid_create(nx, ny)
        sw_elliptic_set_coeffs(g, *[torch.as_tensor(P[k], device="cuda") for k in COEFF_KEYS])
        for R in rhs[p]:
            Rd = torch.as_tensor(R, dtype=torch.float64, device="cuda")
            phi = torch.zeros_like(Rd)
            st = sw_gcr_solve(g, opts, Rd, phi)
            if st.status != SW_OK:
                raise RuntimeError(f"training solve failed: {st.as_dict()}")
            if target == "p3_error":
                p3 = torch.empty_like(Rd)
                sw_precond_apply(g, popts, Rd, p3)
                phi = phi - p3
            R32 = Rd.float()
            sw_model_features(model, g, R32, x0[q])
            sw_model_target(model, g, R32, phi.float(), tg[q])
            q += 1
    torch.cuda.synchronize()
    return x0, tg


def train(model: Model, x0, target, steps: int, batch: int, lr: float, seed: int = 0,
          weight_decay: float = 0.0, warmup: int = 20, log_every: int = 0):
    """AdamW with linear warm-up and cosine decay of the learning rate over
    `steps` mini-batches drawn without replacement per epoch.  Returns the
    per-step losses (read back every log_every steps, else only the last)."""
    import torch
    rng = np.random.default_rng(seed)
    n = x0.shape[0]
    order = rng.permutation(n)
    pos = 0
    losses = []
    for s in range(steps):
        if pos + batch > n:
            order, pos = rng.permutation(n), 0
        idx = torch.as_tensor(order[pos:pos + batch], device="cuda")
        pos += batch
        xb = x0.index_select(0, idx).contiguous()
        tb = target.index_select(0, idx).contiguous()
        f = min(1.0, (s + 1) / max(warmup, 1)) * 0.5 * (1.0 + math.cos(math.pi * s / max(steps, 1)))
        want = (log_every and s % log_every == 0) or s == steps - 1
        loss = sw_model_train_step(model, xb, tb, lr=lr * f, weight_decay=weight_decay, want_loss=bool(want))
        if want:
            losses.append((s, loss))
    return losses


LAYERS = ((4, 32), (32, 64), (64, 64), (128, 64), (96, 32), (32, 1))   # (in, out) channels per 3x3 layer


def init_params(seed: int) -> np.ndarray:
    """He-normal weights and zero biases, flat in the library's order (per
    layer the weights [out][in][3][3], then the biases)."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in LAYERS:
        parts.append((rng.standard_normal((co, ci, 3, 3)) * math.sqrt(2.0 / (9 * ci))).ravel())
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def train_flops_per_point() -> float:
    """Algorithmic FLOPs of one training step per grid point of a sample:
    forward, input gradients of layers 2..6, weight gradients of all layers
    (unpadded channels; 2 FLOPs per multiply-add)."""
    level = (0, 1, 2, 1, 0, 0)
    per = [2.0 * 9 * ci * co / 4 ** l for (ci, co), l in zip(LAYERS, level)]
    return sum(per) + sum(per[1:]) + sum(per)
