"""Parity of the time stepper (sw_swe_*, Eqs. 1-10) with the oracle's
(oracle/swe.py), through the C ABI.

* The explicit part (steps 1-5: transport, forcing, coefficients, right-hand
  side of the increment solve) agrees with the oracle's to rounding: 1e-12 of
  each coefficient field's largest value, and, for R', 64 units in the last
  place of the largest term it is made of, |C Phi^n| (R' is their difference,
  a few hundred times smaller; the cancellation is exact in both).
* Whole steps with FP64 solves at tol 1e-12 on both sides agree to the
  solves' accuracy; with the mixed FP16 solver at tol 1e-8 the increments
  agree to 1e-6 of their size (the solver's parity bar, compounded over the
  steps).
* At the benchmark's size (512 x 256) one FP64 step matches the oracle, and
  over mixed steps the mass changes by no more than the solves' residuals
  allow, a bound that holds at any size.
* Each step solves twice (predictor Phi* = Phi^n, then corrector with the
  predictor's Phi^{n+1}); both passes are checked (the explicit part with a
  given predictor, the stats of both solves).
Grids: several 128-longitude blocks per row with a ragged tail (nx = 320),
nx not a multiple of 4 (66: the scalar operator path), ny odd.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth
from oracle.swe import Stepper

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16120_gb300 as sw  # noqa: E402

A = 6.371e6


def dev(a):
    return None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.cpu().numpy()


def setup(nx, ny, seed, dt=None, orography=500.0, history=True):
    dt = synth.paper_dt(ny) if dt is None else dt
    s = synth.perturbed_state(nx, ny, seed, dt=dt, orography=orography)
    u, v = s.qx / s.phi, s.qy / s.phi
    hist = (0.97 * u + 0.3, 0.95 * v - 0.2) if history else (None, None)
    g = sw.sw_grid_create(nx, ny)
    m = sw.sw_swe_create(g, dt)
    sw.sw_swe_set_state(m, dev(s.phi), dev(s.qx), dev(s.qy), dev(s.h0), dev(s.alpha), dev(s.qbar_x),
                        dev(s.qbar_y))
    if history:
        sw.sw_swe_set_history(m, dev(hist[0]), dev(hist[1]))
    st = Stepper(nx, ny, dt, h0=s.h0, alpha=s.alpha, qbar_x=s.qbar_x, qbar_y=s.qbar_y)
    return s, hist, g, m, st


def state(m):
    ny, nx = m.grid.ny, m.grid.nx
    out = [torch.empty((ny, nx), dtype=torch.float64, device="cuda") for _ in range(3)]
    sw.sw_swe_get_state(m, *out)
    torch.cuda.synchronize()
    return [host(t) for t in out]


def maxrel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("nx,ny,seed,history,given", [(64, 32, 1, True, False), (66, 33, 2, False, True),
                                                      (320, 97, 3, True, True)])
def test_explicit_part_matches_oracle(nx, ny, seed, history, given):
    s, hist, g, m, st = setup(nx, ny, seed, history=history)
    K = [torch.empty((ny, nx), dtype=torch.float64, device="cuda") for _ in range(7)]
    R = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    # the corrector pass's predictor: Phi^n plus a smooth increment of a few metres
    pstar = s.phi + 3.0 * np.cos(synth.grid_coords(nx, ny)[1])[:, None] ** 2 if given else None
    sw.sw_swe_explicit(m, dev(pstar), K, R)
    torch.cuda.synchronize()
    ctx = st.explicit(s.phi, s.qx, s.qy, *hist, phi_star=pstar)
    for k, t in zip(sw.COEFF_KEYS, K):
        assert maxrel(host(t), ctx["coeffs"][k]) <= 1e-12, k
    big = np.max(np.abs(ctx["coeffs"]["C"] * s.phi))
    err = np.max(np.abs(host(R) - ctx["rhs"]))
    assert err <= 64 * np.finfo(np.float64).eps * big
    assert np.max(np.abs(ctx["rhs"])) > 1e3 * err
    # the stepper left the grid holding these coefficients: L(Phi^n) agrees
    y = torch.empty_like(R)
    sw.sw_operator_apply(g, dev(s.phi), y)
    torch.cuda.synchronize()
    assert maxrel(host(y), ctx["problem"].operator(s.phi)) <= 1e-12


@pytest.mark.parametrize("nx,ny,seed", [(64, 32, 4), (66, 33, 5), (320, 97, 6)])
def test_fp64_steps_match_oracle(nx, ny, seed):
    nsteps = 4
    s, hist, g, m, st = setup(nx, ny, seed)
    o = sw.sw_solve_opts_default(prec=sw.SW_PREC_FP64, tol=1e-12, max_iters=3000)
    stats = sw.sw_swe_step(m, o, nsteps)
    assert len(stats) == 2 * nsteps and all(x.converged == 1 and x.status == 0 for x in stats)
    p, qx, qy = s.phi, s.qx, s.qy
    up, vp = hist
    for _ in range(nsteps):
        p, qx, qy, up, vp, info = st.step(p, qx, qy, up, vp, O.Opts(tol=1e-12, max_iters=3000))
    gp, gqx, gqy = state(m)
    assert maxrel(gp - s.phi, p - s.phi) <= 1e-9
    assert maxrel(gqx, qx) <= 1e-10 and maxrel(gqy, qy) <= 1e-9


@pytest.mark.parametrize("prec", [sw.SW_PREC_MIXED_FP16, sw.SW_PREC_MIXED_BF16])
def test_mixed_steps_match_oracle(prec):
    nx, ny, nsteps = 128, 64, 4
    s, hist, g, m, st = setup(nx, ny, 8)
    o = sw.sw_solve_opts_default(prec=prec, tol=1e-8)
    stats = sw.sw_swe_step(m, o, nsteps)
    assert all(x.converged == 1 and x.true_rel_residual <= 1e-8 for x in stats)
    p, qx, qy = s.phi, s.qx, s.qy
    up, vp = hist
    for _ in range(nsteps):
        p, qx, qy, up, vp, _ = st.step(p, qx, qy, up, vp)
    gp, gqx, gqy = state(m)
    assert maxrel(gp - s.phi, p - s.phi) <= 1e-6
    assert maxrel(gqx, qx) <= 1e-6 and maxrel(gqy, qy) <= 1e-6


def test_balanced_flow_matches_oracle():
    nx, ny, dt = 128, 64, 800.0
    s = synth.balanced_zonal_state(nx, ny)
    g = sw.sw_grid_create(nx, ny)
    m = sw.sw_swe_create(g, dt)
    sw.sw_swe_set_state(m, dev(s.phi), dev(s.qx), dev(s.qy))
    stats = sw.sw_swe_step(m, sw.sw_solve_opts_default(prec=sw.SW_PREC_FP64, tol=1e-12, max_iters=3000), 10)
    assert all(x.converged for x in stats)
    p, _, qy, _ = Stepper(nx, ny, dt).run(s.phi, s.qx, s.qy, 10)
    gp, _, gqy = state(m)
    drift_gpu = np.max(np.abs(gp - s.phi))
    drift_or = np.max(np.abs(p - s.phi))
    assert abs(drift_gpu - drift_or) <= 1e-6 * drift_or
    assert maxrel(gqy, qy) <= 1e-8


def test_bench_size_step_and_mass_bound():
    nx, ny = 512, 256
    dt = synth.paper_dt(ny)
    s, hist, g, m, st = setup(nx, ny, 11, history=False)
    o64 = sw.sw_solve_opts_default(prec=sw.SW_PREC_FP64, tol=1e-10, max_iters=3000)
    stats = sw.sw_swe_step(m, o64, 1)
    assert stats[0].converged == 1 and stats[1].converged == 1
    # the corrector starts from the predictor's increment: a fraction of its iterations
    assert stats[1].iterations < stats[0].iterations
    p, qx, qy, _, _, _ = st.step(s.phi, s.qx, s.qy, None, None, O.Opts(tol=1e-10, max_iters=3000))
    gp, gqx, gqy = state(m)
    assert maxrel(gp - s.phi, p - s.phi) <= 1e-7
    assert maxrel(gqx, qx) <= 1e-8 and maxrel(gqy, qy) <= 1e-7
    # mixed steps: the mass sum_ij cos(phi_j) Phi_ij changes only by the solves'
    # residuals, |sum r| <= sqrt(N) ||r||, scaled by dt/2 / a^2 (C = a^2 cos / (dt/2))
    cw = np.cos(synth.grid_coords(nx, ny)[1])[:, None]
    m0 = float(np.sum(cw * gp))
    nsteps = 6
    stats = sw.sw_swe_step(m, sw.sw_solve_opts_default(prec=sw.SW_PREC_MIXED_FP16, tol=1e-8), nsteps)
    assert all(x.converged == 1 for x in stats)
    # from the third step on, the predictor starts from the extrapolated increment
    pred = [x.iterations for x in stats[0::2]]
    assert np.mean(pred[2:]) < pred[0]
    gp2, _, _ = state(m)
    # the corrector's increment is the one applied
    bound = sum(math.sqrt(nx * ny) * x.true_rel_residual * x.R_norm for x in stats[1::2]) * (0.5 * dt) / A ** 2
    assert abs(float(np.sum(cw * gp2)) - m0) <= 1.01 * bound + 1e-13 * m0
    assert np.all(np.isfinite(gp2)) and np.min(gp2) > 0


def test_step_argument_errors():
    g = sw.sw_grid_create(16, 8)
    m = sw.sw_swe_create(g, 600.0)
    o = sw.sw_solve_opts_default()
    with pytest.raises(sw.SwError) as e:
        sw.sw_swe_step(m, o, 1)
    assert e.value.status == sw.SW_ERR_INVALID_ARG
    with pytest.raises(sw.SwError):
        sw.sw_swe_create(g, -1.0)
    z = torch.ones((8, 16), dtype=torch.float64, device="cuda")
    sw.sw_swe_set_state(m, z * 8000.0, 0 * z, 0 * z)
    with pytest.raises(sw.SwError):
        sw.sw_swe_step(m, o, 0)
    with pytest.raises(sw.SwError):
        sw.sw_swe_step(m, sw.sw_solve_opts_default(pc=sw.SW_PC_LEARNED), 1)


def test_full_size_steps_keep_mass_and_stay_bounded():
    """2048 x 1024 (the largest benchmark grid), three mixed steps at the
    paper's scaling of dt (50 s): mass moves only within the solves' residual
    bound, the state stays finite and positive, and the advective Courant
    number stays below 1 on every row, pole rows included."""
    nx, ny = 2048, 1024
    dt = synth.paper_dt(ny)
    s = synth.perturbed_state(nx, ny, 77, dt=dt, orography=500.0)
    g = sw.sw_grid_create(nx, ny)
    m = sw.sw_swe_create(g, dt)
    sw.sw_swe_set_state(m, dev(s.phi), dev(s.qx), dev(s.qy), dev(s.h0), dev(s.alpha), dev(s.qbar_x),
                        dev(s.qbar_y))
    stats = sw.sw_swe_step(m, sw.sw_solve_opts_default(prec=sw.SW_PREC_MIXED_FP16, tol=1e-8, max_iters=2000), 3)
    assert all(x.converged == 1 and x.true_rel_residual <= 1e-8 for x in stats)
    p, qx, qy = state(m)
    assert np.all(np.isfinite(p)) and np.min(p) > 0 and np.all(np.isfinite(qx)) and np.all(np.isfinite(qy))
    lam, phi, dlam, dphi = synth.grid_coords(nx, ny)
    cw = np.cos(phi)[:, None]
    bound = sum(math.sqrt(nx * ny) * x.true_rel_residual * x.R_norm for x in stats[1::2]) * (0.5 * dt) / A ** 2
    m0 = float(np.sum(cw * s.phi))
    assert abs(float(np.sum(cw * p)) - m0) <= 1.01 * bound + 1e-13 * m0
    courant = np.max(np.abs(qx / p) / cw) * dt / (A * dlam)
    assert courant < 1.0
