"""Pins of the time-stepping oracle (oracle/swe.py, Eqs. 1-10).

Each test checks the oracle against something other than its own formulas:

* a solid-body zonal flow over its geostrophically balanced surface is a
  steady solution of Eqs. 1-5; the oracle keeps it steady up to its spatial
  truncation, which falls at second order when the spacing halves;
* a small zonally symmetric bump on fluid at rest (no rotation) oscillates as
  a gravity wave of frequency sqrt(g H l (l+1)) / a; the trapezoidal rule of
  Eq. 6 turns omega dt into 2 atan(omega dt / 2) per step;
* total mass is conserved (flux form of Eq. 1, the increment solved tightly);
* the recovered momenta satisfy the implicit momentum equation, Eqs. 4-6 and 7
  written out here in the metric-coefficient notation of Sec. 2.1 (h_x, h_y,
  G) rather than the oracle's folded Coriolis parameter;
* the coefficients of Eq. 10 are the linear response of the recovered mass
  flux to Phi^{n+1} (the Schur complement of Sec. 2.2), and the right-hand side
  is the trapezoidal Eq. 1 with that flux;
* donor-cell transport at Courant number 1 under a solid-body zonal rotation
  is an exact shift by one cell; in a meridional flow a one-cell spike moves
  only into the downstream cell, by the donor-cell flux;
* white noise on fluid at rest stays bounded at the paper's time step, and fluid
  at rest over a flat bottom does not change in any bit.

With these, a dropped term, a wrong sign or factor of the 2x2 inversion, the
coefficients, the right-hand side or the transport fails at least one pin (each
was checked by planting the mistake in a copy of the oracle).
"""
import math

import numpy as np
import pytest

import synth
from oracle import Opts
from oracle.swe import Stepper, mass

A, OMEGA, G = 6.371e6, 7.292e-5, 9.80616


# derivatives restated for the checks: centred, periodic in longitude, the
# pole row shifted by half a circle beyond each pole
def d_lam(f, dlam):
    return (np.roll(f, -1, 1) - np.roll(f, 1, 1)) / (2 * dlam)


def d_phi(f, dphi):
    nx = f.shape[1]
    below = np.vstack([np.roll(f[0], nx // 2)[None], f[:-1]])
    above = np.vstack([f[1:], np.roll(f[-1], nx // 2)[None]])
    return (above - below) / (2 * dphi)


def geometry(nx, ny):
    _, phi, dlam, dphi = synth.grid_coords(nx, ny)
    hx = (A * np.cos(phi))[:, None]          # h_x = a cos(phi)
    hy = A                                   # h_y = a
    dhx_dy = (-A * np.sin(phi))[:, None]     # d h_x / d phi
    return phi, dlam, dphi, hx, hy, dhx_dy


def forcing(st, Phi, Phi_pg, H0, Qx, Qy, u_metric, alpha, qbx, qby, omega=OMEGA):
    """R_x, R_y of Eqs. 4-5 with the pressure-gradient term given as
    (Phi grad H) components in Phi_pg, the metric force with the zonal wind
    factor u_metric (one momentum factor Q/Phi replaced by it)."""
    _, _, _, hx, hy, dhx_dy = geometry(st.nx, st.ny)
    Gj = hx * hy
    f = 2 * omega * np.sin(geometry(st.nx, st.ny)[0])[:, None]
    pgx, pgy = Phi_pg
    # (1/(G Phi)) (Q_y dh_y/dx - Q_x dh_x/dy) Q_y with dh_y/dx = 0 and Q_x/Phi -> u_metric
    met = -(u_metric * dhx_dy) / Gj
    Rx = -(G / hx) * pgx + f * Qy + met * Qy - alpha * (Qx - qbx)
    Ry = -(G / hy) * pgy - f * Qx - met * Qx - alpha * (Qy - qby)
    return Rx, Ry


def test_balanced_zonal_flow_stays_steady():
    drift, qy = [], []
    for nx, ny in ((64, 32), (128, 64), (256, 128)):
        s = synth.balanced_zonal_state(nx, ny)
        st = Stepper(nx, ny, 300.0)
        p, _, q, infos = st.run(s.phi, s.qx, s.qy, 10)
        assert all(i.stats["converged"] for i in infos)
        drift.append(np.max(np.abs(p - s.phi)))
        qy.append(np.max(np.abs(q)))
    span = np.ptp(synth.balanced_zonal_state(256, 128).phi)   # ~960 m of balanced slope
    assert drift[-1] <= 5e-5 * span
    # second order in the spacing
    assert drift[0] / drift[1] >= 2.8 and drift[1] / drift[2] >= 2.8
    assert qy[0] / qy[1] >= 3.5 and qy[1] / qy[2] >= 3.5


def _mode_phase(nx, ny, dt, degree, nsteps, H=8000.0):
    s = synth.gravity_mode_state(nx, ny, degree, amp=1.0, H=H)
    st = Stepper(nx, ny, dt, omega=0.0)
    _, phi, _, _ = synth.grid_coords(nx, ny)
    P = np.polynomial.legendre.legval(np.sin(phi), [0.0] * degree + [1.0])[:, None]
    w = np.cos(phi)[:, None] * P
    amp = lambda p: np.sum(w * (p - H)) / (nx * np.sum(w * P))  # noqa: E731
    seq = [amp(s.phi)]
    p, qx, qy, up, vp = s.phi, s.qx, s.qy, None, None
    for _ in range(nsteps):
        p, qx, qy, up, vp, _ = st.step(p, qx, qy, up, vp)
        seq.append(amp(p))
    a = np.array(seq)
    # a pure mode obeys a(n+1) + a(n-1) = 2 cos(theta) a(n)
    theta = math.acos(np.sum(a[1:-1] * (a[2:] + a[:-2])) / (2 * np.sum(a[1:-1] ** 2)))
    omega = math.sqrt(G * H * degree * (degree + 1)) / A
    return theta / (2 * math.atan(omega * dt / 2)) - 1.0, a


def test_gravity_wave_frequency():
    e64, a64 = _mode_phase(64, 32, 1800.0, 2, 44)
    e128, _ = _mode_phase(128, 64, 1800.0, 2, 44)
    assert abs(e64) <= 0.01 and abs(e128) <= 0.003
    assert abs(e64) / abs(e128) >= 3.0
    # neutral to within the weak damping of the predictor
    assert 0.98 <= np.max(np.abs(a64[-12:])) <= 1.0 + 1e-9


def test_mass_is_conserved():
    s = synth.perturbed_state(64, 32, 3, orography=500.0)
    st = Stepper(64, 32, 600.0, h0=s.h0, alpha=s.alpha, qbar_x=s.qbar_x, qbar_y=s.qbar_y)
    p, _, _, infos = st.run(s.phi, s.qx, s.qy, 5)
    assert all(i.stats["converged"] for i in infos)
    cw = np.cos(synth.grid_coords(64, 32)[1])[:, None]
    assert abs(mass(p, cw) - mass(s.phi, cw)) <= 1e-13 * mass(s.phi, cw)


@pytest.fixture(scope="module")
def one_step():
    nx, ny, dt = 64, 32, 600.0
    s = synth.perturbed_state(nx, ny, 7, dt=dt, orography=800.0)
    st = Stepper(nx, ny, dt, h0=s.h0, alpha=s.alpha, qbar_x=s.qbar_x, qbar_y=s.qbar_y)
    u, v = s.qx / s.phi, s.qy / s.phi
    up, vp = 0.97 * u + 0.3, 0.95 * v - 0.2           # winds of a previous level
    p1, qx1, qy1, _, _, info = st.step(s.phi, s.qx, s.qy, up, vp, Opts(tol=1e-13, max_iters=3000))
    return s, st, up, vp, p1, qx1, qy1, info


def test_momenta_solve_the_implicit_momentum_equation(one_step):
    s, st, up, vp, p1, qx1, qy1, info = one_step
    ctx = info.ctx
    _, dlam, dphi, _, _, _ = geometry(st.nx, st.ny)
    ps, h0 = ctx["phi_star"], s.h0
    # Eq. 7: (Phi grad H)^{n+1} = (Phi^{n+1} grad(Phi* + H0) + Phi* grad(Phi^{n+1} + H0)) / 2
    pg = (0.5 * (p1 * d_lam(ps + h0, dlam) + ps * d_lam(p1 + h0, dlam)),
          0.5 * (p1 * d_phi(ps + h0, dphi) + ps * d_phi(p1 + h0, dphi)))
    ustar = 2 * s.qx / s.phi - up                     # metric wind extrapolated to n+1
    Rx, Ry = forcing(st, p1, pg, h0, qx1, qy1, ustar, s.alpha, s.qbar_x, s.qbar_y)
    delta = 0.5 * st.dt
    # Eq. 6: Q^{n+1} = Q^ + dt/2 R^{n+1}
    for q1, qh, R in ((qx1, ctx["qhx"], Rx), (qy1, ctx["qhy"], Ry)):
        assert np.max(np.abs(q1 - (qh + delta * R))) <= 1e-12 * np.max(np.abs(q1))


def test_coefficients_are_the_flux_response(one_step):
    s, st, up, vp, p1, qx1, qy1, info = one_step
    ctx, K = info.ctx, info.coeffs
    _, dlam, dphi, hx, hy, _ = geometry(st.nx, st.ny)
    psi = np.random.default_rng(3).standard_normal(p1.shape)
    ax, ay = st.recover(p1, ctx)
    bx, by = st.recover(p1 + psi, ctx)
    # mass flux F = (h_y Q_x, h_x Q_y) (Eq. 1 with Eq. 6's advective velocity)
    fx = hy * (bx - ax)
    fy = hx * (by - ay)
    ex = -(K["A11"] * d_lam(psi, dlam) + K["A12"] * d_phi(psi, dphi) + K["B1"] * psi)
    ey = -(K["A21"] * d_lam(psi, dlam) + K["A22"] * d_phi(psi, dphi) + K["B2"] * psi)
    assert np.max(np.abs(fx - ex)) <= 1e-11 * np.max(np.abs(ex))
    assert np.max(np.abs(fy - ey)) <= 1e-11 * np.max(np.abs(ey))
    assert np.allclose(K["C"], (hx * hy) / (0.5 * st.dt), rtol=1e-15, atol=0)


def test_rhs_is_the_trapezoidal_continuity_equation(one_step):
    s, st, up, vp, p1, qx1, qy1, info = one_step
    ctx, K = info.ctx, info.coeffs
    _, dlam, dphi, hx, hy, _ = geometry(st.nx, st.ny)
    # explicit part of the new mass flux: the recovered flux at Phi^{n+1} = 0
    q0x, q0y = st.recover(np.zeros_like(p1), ctx)
    Fx = hy * (s.qx + q0x)
    Fy = hx * (s.qy + q0y)
    # face values: means of the two cells; nothing through the pole faces
    fxf = 0.5 * (Fx + np.roll(Fx, -1, 1))
    fyf = np.zeros((st.ny + 1, st.nx))
    fyf[1:-1] = 0.5 * (Fy[1:] + Fy[:-1])
    div = (fxf - np.roll(fxf, 1, 1)) / dlam + np.diff(fyf, axis=0) / dphi
    Lphi = ctx["problem"].operator(s.phi)
    want = div - K["C"] * s.phi - Lphi
    assert np.max(np.abs(info.rhs - want)) <= 1e-12 * np.max(np.abs(want))
    # and the step solved it: continuity G (Phi^{n+1} - Phi^n) / (dt/2) = -div F^n - div F^{n+1}
    r = ctx["problem"].operator(info.dphi) - info.rhs
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(info.rhs)


def test_donor_cell_transport_is_an_exact_shift_at_courant_one():
    nx, ny, u0 = 64, 32, 20.0
    lam, phi, dlam, dphi = synth.grid_coords(nx, ny)
    c = np.cos(phi)[:, None]
    depth = 8000.0 + 30.0 * np.cos(3 * lam)[None, :] * c ** 2 + 5.0 * np.sin(phi)[:, None]
    u = u0 * c * np.ones((1, nx))
    v = np.zeros((ny, nx))
    qx, qy = depth * u, depth * v
    up = 0.8 * u                                      # U^{n+1/2} = a (1.5 u - 0.5 up) = 1.1 a u
    dt = A * dlam / (1.1 * u0)
    st = Stepper(nx, ny, dt)
    ctx = st.explicit(depth, qx, qy, up, v)
    # Q^ = shift of Q^n + dt/2 R^n, R^n from Eqs. 4-5 at level n
    pg = (depth * d_lam(depth, dlam), depth * d_phi(depth, dphi))
    zero = np.zeros_like(depth)
    Rx, Ry = forcing(st, depth, pg, zero, qx, qy, u, zero, zero, zero)
    delta = 0.5 * dt
    for qh, q, R in ((ctx["qhx"], qx, Rx), (ctx["qhy"], qy, Ry)):
        want = np.roll(q + delta * R, 1, 1)
        assert np.max(np.abs(qh - want)) <= 1e-11 * np.max(np.abs(want))


def test_donor_cell_meridional_transport_reaches_only_downstream():
    """A one-cell momentum spike in a northward flow changes, after one
    donor-cell step, only its own cell and the cell north of it, by the flux
    V_(j+1/2) * spike * dt / dphi leaving one and entering the other.  The
    spike's wind is cancelled in the extrapolated advective velocity
    (u_prev = 3u), so both runs are carried by the same velocity field."""
    nx, ny, v0, dt = 32, 16, 10.0, 600.0
    lam, phi, dlam, dphi = synth.grid_coords(nx, ny)
    depth = np.full((ny, nx), 8000.0)
    qy = depth * v0
    j0, i0, S = 6, 11, 5000.0
    st = Stepper(nx, ny, dt, omega=0.0)
    runs = []
    for spike in (0.0, S):
        qx = np.zeros((ny, nx))
        qx[j0, i0] = spike
        u = qx / depth
        runs.append(st.explicit(depth, qx, qy, 3.0 * u, np.full((ny, nx), v0)))
    delta = 0.5 * dt
    c = np.cos(phi)
    vface = A * v0 * 0.5 * (c[j0] + c[j0 + 1])         # mean of the two cells' a cos(phi) v
    zero = np.zeros((ny, nx))
    qx = zero.copy()
    qx[j0, i0] = S
    Rx, Ry = forcing(st, depth, (zero, zero), zero, qx, qy, qx / depth, zero, zero, zero, omega=0.0)
    Rx0, Ry0 = forcing(st, depth, (zero, zero), zero, zero, qy, zero, zero, zero, zero, omega=0.0)
    for key, s1 in (("qhx", S + delta * (Rx - Rx0)[j0, i0]), ("qhy", delta * (Ry - Ry0)[j0, i0])):
        d = runs[1][key] - runs[0][key]
        moved = vface * s1 * dt / dphi
        want = np.zeros_like(d)
        want[j0, i0] = s1 - moved / (A * A * c[j0])
        want[j0 + 1, i0] = moved / (A * A * c[j0 + 1])
        # the difference of two transported fields: rounding of the larger one
        assert np.max(np.abs(d - want)) <= 1e-12 * max(abs(s1), np.max(np.abs(runs[0][key]))), key


def test_noise_does_not_grow_at_the_papers_time_step():
    """White noise on fluid at rest, at the paper's 800 s step on 128 x 64:
    the external-mode Courant number reaches about 30 on the pole rows, where
    the transport predictor of Eq. 7 amplifies the short zonal waves by one to
    two orders of magnitude per step.  With the outer-iteration predictor the
    noise stays bounded (the trapezoidal gravity waves are neutral, the
    transport damps)."""
    nx, ny, dt, H = 128, 64, 800.0, 8000.0
    rng = np.random.default_rng(12)
    noise = rng.standard_normal((ny, nx))
    st = Stepper(nx, ny, dt)
    p, qx, qy = H + noise, np.zeros((ny, nx)), np.zeros((ny, nx))
    up = vp = None
    for _ in range(30):
        p, qx, qy, up, vp, info = st.step(p, qx, qy, up, vp, Opts(tol=1e-10, max_iters=2000))
        assert info.stats["converged"] == 1
    assert np.max(np.abs(p - H)) <= 1.5 * np.max(np.abs(noise))
    assert np.max(np.abs(qx / p)) < 1.0 and np.max(np.abs(qy / p)) < 1.0


def test_rest_state_is_exactly_steady():
    """Fluid at rest over a flat bottom: every flux vanishes, C Phi^n cancels
    L(Phi^n) exactly, the right-hand side of each solve is zero and the solves
    return zero increments, so the state does not change in any bit."""
    nx, ny, H = 32, 16, 8000.0
    st = Stepper(nx, ny, 800.0)
    p0 = np.full((ny, nx), H)
    z = np.zeros((ny, nx))
    p, qx, qy, infos = st.run(p0, z, z, 3)
    assert all(np.all(i.rhs == 0.0) and i.stats["iterations"] == 0 for i in infos)
    assert np.array_equal(p, p0) and not np.any(qx) and not np.any(qy)
