"""Seeded initial states for the semi-implicit shallow-water time stepping
around the solver (Eqs. 1-8).

A state is the fluid thickness Phi (m) and the momenta Qx = Phi u, Qy = Phi v
(m^2/s, u and v the zonal and meridional winds in m/s) on the collocated
grid, plus the fixed fields of the forcing: orography H0, the relaxation
inverse time scale alpha and the relaxation target (Qbar_x, Qbar_y) of
Eqs. 4-5.

* `balanced_zonal_state`: solid-body zonal flow u = u0 cos(phi), v = 0, over a
  free surface in geostrophic balance with it.  Steady zonal flow needs R_y = 0
  in Eq. 5, i.e. (g/a) d(Phi + H0)/dphi = -(2 Omega sin(phi) + u tan(phi)/a) u;
  with u = u0 cos(phi) this integrates to
      Phi + H0 = H - (a/g) (Omega u0 + u0^2 / (2a)) sin^2(phi).
  Eq. 4 and Eq. 1 hold trivially (no zonal gradients, no meridional flow).
* `gravity_mode_state`: fluid at rest (u = v = 0) of mean depth H with a small
  zonally symmetric Legendre-mode bump.
* `perturbed_state`: the balanced flow plus seeded smooth perturbations of the
  thickness (2 % of H, spherical-harmonic degrees 2..6) and of the winds
  (streamfunction degrees 2..4, at most 15 m/s), optional orography and the
  polar absorber.  Zonal wavenumber 1 is left out of every perturbation:
  flow across a pole, or a wavenumber-1 pressure pattern that drives one,
  makes the zonal wind of the longitude/latitude grid finite at the pole
  rows, where the zonal spacing a cos(phi) dlam is tiny, and the explicit
  advection would break its Courant limit there.  Wavenumbers 0 and >= 2 give
  flows that decay towards the poles, like those of the paper's test cases
  (Sec. 3.1), which is what lets the time step shrink only linearly with the
  grid spacing (800, 400 and 200 s at 128 x 64, 256 x 128 and 512 x 256).

Layout: float64 arrays (ny, nx), as everywhere in this package.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .shallow_water import EARTH, absorber
from .sphere import grid_coords, random_sh_field


@dataclass
class ModelState:
    nx: int
    ny: int
    phi: np.ndarray             # thickness Phi (m)
    qx: np.ndarray              # Phi u (m^2/s)
    qy: np.ndarray              # Phi v (m^2/s)
    h0: np.ndarray | None       # orography (m), None = flat
    alpha: np.ndarray | None    # relaxation inverse time scale (1/s), None = 0
    qbar_x: np.ndarray | None   # relaxation target, None = 0
    qbar_y: np.ndarray | None


def _c(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def balanced_zonal_state(nx: int, ny: int, u0: float = 20.0, H: float = 8000.0,
                         a: float = EARTH["a"], omega: float = EARTH["omega"],
                         g: float = EARTH["g"]) -> ModelState:
    _, phi, _, _ = grid_coords(nx, ny)
    s = np.sin(phi)[:, None]
    c = np.cos(phi)[:, None]
    depth = H - (a / g) * (omega * u0 + u0 * u0 / (2.0 * a)) * s * s
    depth = np.broadcast_to(depth, (ny, nx))
    u = np.broadcast_to(u0 * c, (ny, nx))
    return ModelState(nx, ny, _c(depth), _c(depth * u), np.zeros((ny, nx)), None, None, None, None)


def gravity_mode_state(nx: int, ny: int, degree: int = 2, amp: float = 1.0,
                       H: float = 8000.0) -> ModelState:
    """Rest state of depth H plus amp * P_degree(sin phi) (Legendre polynomial,
    P(1) = 1)."""
    _, phi, _, _ = grid_coords(nx, ny)
    x = np.sin(phi)
    p = np.polynomial.legendre.legval(x, [0.0] * degree + [1.0])
    depth = H + amp * np.broadcast_to(p[:, None], (ny, nx))
    return ModelState(nx, ny, _c(depth), np.zeros((ny, nx)), np.zeros((ny, nx)), None, None, None, None)


def _modes(lmin, lmax, skip_m1):
    return [(l, m) for l in range(lmin, lmax + 1) for m in range(-l, l + 1)
            if not (skip_m1 and abs(m) == 1)]


def paper_dt(ny: int) -> float:
    """The paper's time step for its grids (Sec. 3.1): 800 s at ny = 64, halved
    with every doubling of the resolution."""
    return 800.0 * 64.0 / ny


def perturbed_state(nx: int, ny: int, seed: int, dt: float = 600.0, u0: float = 20.0,
                    H: float = 8000.0, rel_amp: float = 0.02, wmax: float = 15.0,
                    orography: float = 0.0, absorb: bool = True,
                    a: float = EARTH["a"], omega: float = EARTH["omega"],
                    g: float = EARTH["g"]) -> ModelState:
    """Balanced zonal flow plus seeded perturbations (see the module docstring).

    `orography` > 0 adds a smooth mountain field of that maximum height and
    lowers the thickness by it, so that the free surface Phi + H0 keeps the
    balanced shape.  With `absorb` the relaxation is the polar absorber of
    Sec. 3.2 (alpha_max = 1/(200 dt)) towards the initial momenta."""
    lam, phi, dlam, dphi = grid_coords(nx, ny)
    rng = np.random.default_rng(seed)
    base = balanced_zonal_state(nx, ny, u0, H, a, omega, g)
    mh = _modes(2, 6, True)
    dh = random_sh_field(lam, phi, rng.standard_normal(len(mh)), mh)
    dh *= rel_amp * H / np.max(np.abs(dh))
    mp = _modes(2, 4, True)
    cp = rng.standard_normal(len(mp))
    # winds of the streamfunction psi from its exact derivatives: the latitude
    # derivative of each term by a centred difference of the analytic field
    eps = 1e-6
    psi_p = random_sh_field(lam, phi + eps, cp, mp)
    psi_m = random_sh_field(lam, phi - eps, cp, mp)
    dpsi_dphi = (psi_p - psi_m) / (2.0 * eps)
    lam_p = random_sh_field(lam + eps, phi, cp, mp)
    lam_m = random_sh_field(lam - eps, phi, cp, mp)
    dpsi_dlam = (lam_p - lam_m) / (2.0 * eps)
    cphi = np.cos(phi)[:, None]
    du = -dpsi_dphi
    dv = dpsi_dlam / cphi
    ws = wmax / max(np.max(np.abs(du)), np.max(np.abs(dv)))
    u = base.qx / base.phi + ws * du
    v = ws * dv
    depth = base.phi + dh
    h0 = None
    if orography > 0.0:
        mo = _modes(2, 5, True)
        hm = random_sh_field(lam, phi, rng.standard_normal(len(mo)), mo)
        hm = orography * (hm - hm.min()) / (hm.max() - hm.min())
        h0 = _c(hm)
        depth = depth - hm
    qx = depth * u
    qy = depth * v
    alpha = None
    if absorb:
        alpha = _c(np.broadcast_to(absorber(phi, 1.0 / (200.0 * dt))[:, None], (ny, nx)))
    return ModelState(nx, ny, _c(depth), _c(qx), _c(qy), h0, alpha,
                      _c(qx.copy()) if absorb else None, _c(qy.copy()) if absorb else None)
