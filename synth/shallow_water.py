"""Synthetic shallow-water states -> coefficients and right-hand side of the
semi-implicit Helmholtz problem (Eqs. 1-10).

The paper's own test cases (Rossby-Haurwitz wave 4, zonal flow over Earth
orography, Sec. 3) need initial conditions and an orography data set that are
not available here; seeded smooth states of the same shape stand in for them:

* depth  Phi* = H0 + h,  h a random spherical-harmonic sum with total
  wavenumber 1..8, scaled so that max|h| = 5% of H0 (H0 = 8000 m);
* winds from a random streamfunction with wavenumbers 1..4,
  u = -(1/a) dpsi/dphi,  v = (1/(a cos phi)) dpsi/dlam,  scaled to max 40 m/s;
* weak polar absorber (Sec. 3.2): alpha rises linearly from 0 at an angular
  distance 3*pi/64 from a pole to alpha_max = 1/(200 dt) at the pole.

Coefficients of the generalised Laplacian (Eq. 10).  The paper only says they
are straightforward modifications of those of the closed-form momentum
expression (Eq. 8); written out from Eqs. 1-8 they read (delta = dt/2,
f = 2 Omega sin phi, the metric force folded into the Coriolis parameter
f~ = f + u tan(phi)/a, c = 1 + delta*alpha, b = delta*f~, D = c^2 + b^2,
kappa = delta*g*Phi*/2, H* = Phi* + H0 with flat orography H0 = 0):

  A11 =  kappa c / (D cos phi)     A12 = kappa b / D
  A21 = -kappa b / D               A22 = kappa c cos phi / D
  B1  = (delta g / 2D) (c dH*/dlam / cos phi + b dH*/dphi)
  B2  = (delta g / 2D) (c cos phi dH*/dphi - b dH*/dlam)
  C   = a^2 cos phi / delta        (the Jacobian G = a^2 cos phi over delta)

Right-hand side: the discrete divergence of a seeded smooth face-centred
vector field whose meridional component vanishes on the pole faces, so that
sum(R) = 0.  Its amplitude a*H0*U with U = 10 m/s gives solutions of a few
metres to tens of metres, the size of a time-step increment.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .sphere import grid_coords, random_sh_field, sh_modes

EARTH = dict(a=6.371e6, omega=7.292e-5, g=9.80616)


@dataclass
class SWState:
    nx: int
    ny: int
    phi_star: np.ndarray  # depth predictor Phi*, (ny, nx)
    u: np.ndarray         # zonal wind, (ny, nx)
    v: np.ndarray         # meridional wind, (ny, nx)


def _ddlam(f: np.ndarray, dlam: float) -> np.ndarray:
    return (np.roll(f, -1, axis=1) - np.roll(f, 1, axis=1)) / (2.0 * dlam)


def _ddphi(f: np.ndarray, dphi: float) -> np.ndarray:
    """Centred meridional difference; the row beyond a pole is the pole row
    shifted by half a circle (the same physical points across the pole)."""
    nx = f.shape[1]
    south = np.roll(f[0], nx // 2)[None, :]
    north = np.roll(f[-1], nx // 2)[None, :]
    ext = np.concatenate([south, f, north], axis=0)
    return (ext[2:] - ext[:-2]) / (2.0 * dphi)


def synthetic_state(nx: int, ny: int, seed: int, theta: float = 0.0,
                    H0: float = 8000.0, rel_amp: float = 0.05,
                    umax: float = 40.0, a: float = EARTH["a"]) -> SWState:
    """Seeded smooth state.  `theta` moves the state along a smooth periodic
    path: two i.i.d. normal coefficient sets cA, cB are blended as
    cA cos(theta) + cB sin(theta), which keeps the statistics unchanged; the
    scale factors are fixed at theta = 0 so amplitudes stay bounded."""
    lam, phi, dlam, dphi = grid_coords(nx, ny)
    rng = np.random.default_rng(seed)
    mh = sh_modes(1, 8)
    mp = sh_modes(1, 4)
    ch_a = rng.standard_normal(len(mh))
    ch_b = rng.standard_normal(len(mh))
    cp_a = rng.standard_normal(len(mp))
    cp_b = rng.standard_normal(len(mp))
    h0 = random_sh_field(lam, phi, ch_a, mh)
    hs = rel_amp * H0 / np.max(np.abs(h0))
    h = hs * random_sh_field(lam, phi, ch_a * math.cos(theta) + ch_b * math.sin(theta), mh)
    psi0 = random_sh_field(lam, phi, cp_a, mp)
    cphi = np.cos(phi)[:, None]
    u0 = -_ddphi(psi0, dphi) / a
    v0 = _ddlam(psi0, dlam) / (a * cphi)
    ws = umax / max(np.max(np.abs(u0)), np.max(np.abs(v0)))
    psi = random_sh_field(lam, phi, cp_a * math.cos(theta) + cp_b * math.sin(theta), mp)
    u = -ws * _ddphi(psi, dphi) / a
    v = ws * _ddlam(psi, dlam) / (a * cphi)
    return SWState(nx, ny, H0 + h, u, v)


def absorber(phi: np.ndarray, alpha_max: float) -> np.ndarray:
    """Polar absorber inverse time scale (Sec. 3.2): linear ramp from 0 at an
    angular distance 3*pi/64 from the nearer pole to alpha_max at the pole."""
    d = 0.5 * math.pi - np.abs(phi)
    return alpha_max * np.maximum(0.0, 1.0 - d / (3.0 * math.pi / 64.0))


def coefficients(state: SWState, dt: float = 600.0, alpha_max: float | None = None,
                 a: float = EARTH["a"], omega: float = EARTH["omega"],
                 g: float = EARTH["g"]) -> dict:
    """Coefficient fields of Eq. 10 for the given state (formulas in the module
    docstring).  Returns float64 arrays A11, A12, A21, A22, B1, B2, C."""
    nx, ny = state.nx, state.ny
    lam, phi, dlam, dphi = grid_coords(nx, ny)
    if alpha_max is None:
        alpha_max = 1.0 / (200.0 * dt)
    delta = 0.5 * dt
    cphi = np.cos(phi)[:, None]
    sphi = np.sin(phi)[:, None]
    f = 2.0 * omega * sphi
    ftil = f + state.u * (sphi / cphi) / a
    c = np.broadcast_to(1.0 + delta * absorber(phi, alpha_max)[:, None], (ny, nx))
    b = delta * ftil
    D = c * c + b * b
    kappa = 0.5 * delta * g * state.phi_star
    hstar = state.phi_star
    dhl = _ddlam(hstar, dlam)
    dhp = _ddphi(hstar, dphi)
    out = {
        "A11": kappa * c / (D * cphi),
        "A12": kappa * b / D,
        "A21": -kappa * b / D,
        "A22": kappa * c * cphi / D,
        "B1": (0.5 * delta * g / D) * (c * dhl / cphi + b * dhp),
        "B2": (0.5 * delta * g / D) * (c * cphi * dhp - b * dhl),
        "C": np.broadcast_to(a * a * cphi / delta, (ny, nx)).copy(),
    }
    return {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in out.items()}


def rhs_divergence(nx: int, ny: int, seed: int, theta: float = 0.0,
                   H0: float = 8000.0, U: float = 10.0,
                   a: float = EARTH["a"]) -> np.ndarray:
    """R = discrete flux divergence of a seeded smooth face-centred vector
    field (F^lam at (i+1/2, j), F^phi at (i, j+1/2), F^phi = 0 on pole faces)."""
    lam, phi, dlam, dphi = grid_coords(nx, ny)
    rng = np.random.default_rng(seed + 7919)
    modes = sh_modes(1, 6)
    s1a, s1b = rng.standard_normal(len(modes)), rng.standard_normal(len(modes))
    s2a, s2b = rng.standard_normal(len(modes)), rng.standard_normal(len(modes))
    ct, st = math.cos(theta), math.sin(theta)
    lam_f = lam + 0.5 * dlam
    phi_f = phi[:-1] + 0.5 * dphi
    s1 = random_sh_field(lam_f, phi, s1a, modes)
    s2 = np.cos(phi_f)[:, None] * random_sh_field(lam, phi_f, s2a, modes)
    scale = a * H0 * U / max(np.max(np.abs(s1)), np.max(np.abs(s2)))
    fl = scale * random_sh_field(lam_f, phi, s1a * ct + s1b * st, modes)
    fp_in = scale * np.cos(phi_f)[:, None] * random_sh_field(lam, phi_f, s2a * ct + s2b * st, modes)
    fp = np.zeros((ny + 1, nx))
    fp[1:ny] = fp_in
    div = (fl - np.roll(fl, 1, axis=1)) / dlam + (fp[1:] - fp[:-1]) / dphi
    return np.ascontiguousarray(div, dtype=np.float64)


def problem(nx: int, ny: int, seed: int, dt: float = 600.0, theta: float = 0.0,
            alpha_max: float | None = None) -> dict:
    """One elliptic problem: coefficient fields + R (keys A11..C, R)."""
    st = synthetic_state(nx, ny, seed, theta=theta)
    out = coefficients(st, dt=dt, alpha_max=alpha_max)
    out["R"] = rhs_divergence(nx, ny, seed, theta=theta)
    return out


SEQ_DTHETA = 0.05  # radians per solve along the evolving sequence


def sequence_problem(nx: int, ny: int, seed: int, step: int, dt: float = 600.0) -> dict:
    """Step `step` of a smoothly evolving sequence of problems: the state and
    the right-hand side move along their periodic paths by SEQ_DTHETA per step,
    which changes Phi* by well under 1% between consecutive steps."""
    return problem(nx, ny, seed, dt=dt, theta=step * SEQ_DTHETA)


def ensemble_members(spec=((32, 128, 64), (24, 256, 128), (8, 512, 256)), seed_block: int = 2):
    """(nx, ny, seed) for each member of a batched ensemble; seeds are
    1000*seed_block + member index."""
    out = []
    k = 0
    for count, nx, ny in spec:
        for _ in range(count):
            out.append((nx, ny, 1000 * seed_block + k))
            k += 1
    return out


def random_rhs(nx: int, ny: int, seed: int, n: int) -> np.ndarray:
    """n seeded right-hand sides [n, ny, nx] of unit RMS, from smooth to rough:
    white noise whose 2-D spectrum is damped by (1 + (k / k0)^2)^(-p/2) with a
    random corner k0 (2..nx/4 wavenumbers) and slope p (0..3) per field."""
    rng = np.random.default_rng(seed + 104729)
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.rfftfreq(nx) * nx
    kk = np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)
    out = np.empty((n, ny, nx))
    for q in range(n):
        k0 = math.exp(rng.uniform(math.log(2.0), math.log(nx / 4)))
        p = rng.uniform(0.0, 3.0)
        spec = np.fft.rfft2(rng.standard_normal((ny, nx))) * (1.0 + (kk / k0) ** 2) ** (-p / 2)
        f = np.fft.irfft2(spec, s=(ny, nx))
        out[q] = f / math.sqrt(float(np.mean(f * f)))
    return out
