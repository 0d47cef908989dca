"""Plain FP64 semi-implicit shallow-water time step around the elliptic solve
(Eqs. 1-10, Sec. 2.2).  Test infrastructure only: the product path never
imports this module.

One step n -> n+1, in the order of Sec. 2.2, numpy float64 on (ny, nx) arrays:

1. winds u = Qx/Phi, v = Qy/Phi at level n (Eq. 6 gives the advective
   velocity G(x', y') = (a u, a cos(phi) v)); its value at n + 1/2 by linear
   extrapolation from n and n-1;
2. the explicit forcing R^n of Eqs. 4-5 (pressure gradient, Coriolis and
   metric force, relaxation), and Q^ = M(Q^n + dt/2 R^n) of Eq. 6;
3. for a thickness predictor Phi*: the coefficient fields of Eq. 10 at n+1
   (Eq. 7's pressure gradient, Coriolis and relaxation implicit, the metric
   force folded into the Coriolis parameter f~ = f + u* tan(phi)/a, u* the
   zonal wind extrapolated to n+1; the 2x2 system of Eq. 8 inverted in closed
   form);
4. the right-hand side: the trapezoidal Eq. 1 with the momenta of Eq. 8
   gives L(Phi^{n+1}) = div(F^n + F0) - (G/delta) Phi^n, F = (a Qx, a cos(phi) Qy)
   the mass flux and F0 its explicit part at n+1; solved for the increment,
   L(dPhi) = that - L(Phi^n), so the solver's relative residual is the
   paper's ||r|| / ||r0|| with first guess Phi^n (Sec. 2.3);
5. steps 3-4 run twice: first with Phi* = Phi^n (increment from zero), then
   with Phi* = the Phi^{n+1} of the first solve (increment warm-started from
   the first one) -- one outer iteration in place of the explicit transport
   predictor of Eq. 7, which is unstable at the external-mode Courant numbers
   of the pole rows (the reading and its von Neumann analysis are recorded
   with the design);
6. Phi^{n+1} = Phi^n + dPhi and the momenta from Eq. 8.

The explicit transport M is first-order donor-cell upwinding in flux form
(MPDATA itself is outside this build).  Derivatives at cell centres are
centred differences, periodic in longitude, with the pole row shifted by half
a circle as the row beyond a pole.  The flux divergence of step 4 takes face
values as means of the two adjacent cells and no meridional flux through the
pole faces, as the operator of Eq. 10 does.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .oracle import Opts, Problem

EARTH_A, EARTH_OMEGA, EARTH_G = 6.371e6, 7.292e-5, 9.80616


def _ddlam(f, dlam):
    return (np.roll(f, -1, axis=1) - np.roll(f, 1, axis=1)) / (2.0 * dlam)


def _ddphi(f, dphi):
    nx = f.shape[1]
    ext = np.concatenate([np.roll(f[:1], nx // 2, axis=1), f, np.roll(f[-1:], nx // 2, axis=1)])
    return (ext[2:] - ext[:-2]) / (2.0 * dphi)


@dataclass
class StepInfo:
    ctx: dict                # every intermediate field of the explicit part (second pass)
    dphi: np.ndarray         # the increment solved for (second pass)
    stats: dict              # second solve
    stats1: dict             # first solve (Phi* = Phi^n)
    dphi1: np.ndarray        # its increment

    @property
    def phi_star(self):
        return self.ctx["phi_star"]

    @property
    def coeffs(self):
        return self.ctx["coeffs"]

    @property
    def rhs(self):
        return self.ctx["rhs"]


class Stepper:
    """Time stepping of Eqs. 1-8 with the elliptic solve of Eqs. 9-10."""

    def __init__(self, nx: int, ny: int, dt: float, a: float = EARTH_A, omega: float = EARTH_OMEGA,
                 g: float = EARTH_G, h0=None, alpha=None, qbar_x=None, qbar_y=None):
        self.nx, self.ny, self.dt, self.a, self.omega, self.g = nx, ny, float(dt), a, omega, g
        self.dlam = 2.0 * math.pi / nx
        self.dphi = math.pi / ny
        lat = -0.5 * math.pi + (np.arange(ny) + 0.5) * self.dphi
        self.cos = np.cos(lat)[:, None]
        self.sin = np.sin(lat)[:, None]
        self.tan = self.sin / self.cos
        z = np.zeros((ny, nx))
        self.h0 = z if h0 is None else np.asarray(h0, dtype=np.float64)
        self.alpha = z if alpha is None else np.asarray(alpha, dtype=np.float64)
        self.qbx = z if qbar_x is None else np.asarray(qbar_x, dtype=np.float64)
        self.qby = z if qbar_y is None else np.asarray(qbar_y, dtype=np.float64)

    # -- explicit transport (Eq. 1 / Eq. 6 with donor-cell fluxes) ----------
    def _upwind_div(self, psi, U, V):
        """div(V psi) with donor-cell face fluxes; U, V cell-centred advective
        velocities (a u, a cos(phi) v); face velocity = mean of the two cells,
        zero through the pole faces."""
        Uf = 0.5 * (U + np.roll(U, -1, axis=1))                       # i + 1/2
        Fl = np.maximum(Uf, 0.0) * psi + np.minimum(Uf, 0.0) * np.roll(psi, -1, axis=1)
        Vf = 0.5 * (V[:-1] + V[1:])                                   # j + 1/2, interior faces
        Fp = np.zeros((self.ny + 1, self.nx))
        Fp[1:-1] = np.maximum(Vf, 0.0) * psi[:-1] + np.minimum(Vf, 0.0) * psi[1:]
        return (Fl - np.roll(Fl, 1, axis=1)) / self.dlam + (Fp[1:] - Fp[:-1]) / self.dphi

    def _face_div(self, Fx, Fy):
        """Divergence of cell-centred fluxes through faces holding the mean of
        the two adjacent cells; no meridional flux through the pole faces."""
        fl = 0.5 * (Fx + np.roll(Fx, -1, axis=1))
        fp = np.zeros((self.ny + 1, self.nx))
        fp[1:-1] = 0.5 * (Fy[:-1] + Fy[1:])
        return (fl - np.roll(fl, 1, axis=1)) / self.dlam + (fp[1:] - fp[:-1]) / self.dphi

    def explicit(self, phi, qx, qy, u_prev=None, v_prev=None, phi_star=None) -> dict:
        """Steps 1-4: everything before an elliptic solve.  u_prev, v_prev:
        winds at n-1 (None: those of level n); phi_star: the thickness
        predictor (None: Phi^n).  Returns the intermediate fields by name."""
        a, g, dt = self.a, self.g, self.dt
        delta = 0.5 * dt
        G = a * a * self.cos
        # 1. winds and the advective velocity at n + 1/2
        u = qx / phi
        v = qy / phi
        up = u if u_prev is None else u_prev
        vp = v if v_prev is None else v_prev
        U = a * (1.5 * u - 0.5 * up)
        V = a * self.cos * (1.5 * v - 0.5 * vp)
        if phi_star is None:
            phi_star = phi
        # 2. explicit forcing at n (Eqs. 4-5) and the transported momenta (Eq. 6)
        fn = 2.0 * self.omega * self.sin + u * self.tan / a
        hn = phi + self.h0
        Rx = -(g / (a * self.cos)) * phi * _ddlam(hn, self.dlam) + fn * qy - self.alpha * (qx - self.qbx)
        Ry = -(g / a) * phi * _ddphi(hn, self.dphi) - fn * qx - self.alpha * (qy - self.qby)
        px = qx + delta * Rx
        py = qy + delta * Ry
        qhx = px - (dt / G) * self._upwind_div(px, U, V)
        qhy = py - (dt / G) * self._upwind_div(py, U, V)
        # 3. implicit Coriolis + relaxation at n+1, metric force in f~ (Eq. 8)
        ustar = 2.0 * u - up
        fs = 2.0 * self.omega * self.sin + ustar * self.tan / a
        c = 1.0 + delta * self.alpha
        b = delta * fs
        D = c * c + b * b
        kappa = 0.5 * delta * g * phi_star
        hs = phi_star + self.h0
        dhl = _ddlam(hs, self.dlam)
        dhp = _ddphi(hs, self.dphi)
        coeffs = {
            "A11": kappa * c / (D * self.cos),
            "A12": kappa * b / D,
            "A21": -kappa * b / D,
            "A22": kappa * c * self.cos / D,
            "B1": (0.5 * delta * g / D) * (c * dhl / self.cos + b * dhp),
            "B2": (0.5 * delta * g / D) * (c * self.cos * dhp - b * dhl),
            "C": G / delta,
        }
        coeffs = {k: np.ascontiguousarray(np.broadcast_to(x, phi.shape)) for k, x in coeffs.items()}
        # explicit part of the momenta at n+1: Eq. 7's Phi* grad(H0) term is known
        X0 = qhx + delta * self.alpha * self.qbx - delta * (0.5 * g / (a * self.cos)) * phi_star * _ddlam(self.h0, self.dlam)
        Y0 = qhy + delta * self.alpha * self.qby - delta * (0.5 * g / a) * phi_star * _ddphi(self.h0, self.dphi)
        F0x = a * (c * X0 + b * Y0) / D
        F0y = a * self.cos * (c * Y0 - b * X0) / D
        # 4. right-hand side of the increment solve
        prob = Problem(coeffs)
        rhs = self._face_div(a * qx + F0x, a * self.cos * qy + F0y) - coeffs["C"] * phi - prob.operator(phi)
        return dict(u=u, v=v, U=U, V=V, phi_star=phi_star, Rx=Rx, Ry=Ry, qhx=qhx, qhy=qhy, ustar=ustar,
                    c=c, b=b, D=D, dhl=dhl, dhp=dhp, coeffs=coeffs, X0=X0, Y0=Y0, F0x=F0x, F0y=F0y,
                    rhs=rhs, problem=prob)

    def recover(self, phi1, ctx):
        """Step 6: the momenta at n+1 from Eq. 8 with Eq. 7's pressure gradient."""
        a, g, delta = self.a, self.g, 0.5 * self.dt
        Px = -(0.5 * g / (a * self.cos)) * (phi1 * ctx["dhl"] + ctx["phi_star"] * _ddlam(phi1, self.dlam))
        Py = -(0.5 * g / a) * (phi1 * ctx["dhp"] + ctx["phi_star"] * _ddphi(phi1, self.dphi))
        X = ctx["X0"] + delta * Px
        Y = ctx["Y0"] + delta * Py
        c, b, D = ctx["c"], ctx["b"], ctx["D"]
        return (c * X + b * Y) / D, (c * Y - b * X) / D

    def step(self, phi, qx, qy, u_prev=None, v_prev=None, opts: Opts | None = None):
        """One step (two solves, step 5).  Returns (phi1, qx1, qy1, u_n, v_n,
        StepInfo)."""
        if opts is None:
            opts = Opts(tol=1e-12, max_iters=2000)
        ctx1 = self.explicit(phi, qx, qy, u_prev, v_prev)
        d1, st1 = ctx1["problem"].gcr(ctx1["rhs"], opts)
        ctx = self.explicit(phi, qx, qy, u_prev, v_prev, phi_star=phi + d1)
        dphi, stats = ctx["problem"].gcr(ctx["rhs"], opts, phi0=d1)
        phi1 = phi + dphi
        qx1, qy1 = self.recover(phi1, ctx)
        return phi1, qx1, qy1, ctx["u"], ctx["v"], StepInfo(ctx, dphi, stats, st1, d1)

    def run(self, phi, qx, qy, nsteps: int, opts: Opts | None = None):
        """nsteps steps from a state without history; returns the final state
        and the list of StepInfo."""
        up = vp = None
        infos = []
        for _ in range(nsteps):
            phi, qx, qy, up, vp, info = self.step(phi, qx, qy, up, vp, opts)
            infos.append(info)
        return phi, qx, qy, infos


def mass(phi, cos_lat):
    """Total mass sum_ij cos(phi_j) Phi_ij (the area weight up to a constant)."""
    return float(np.sum(cos_lat * phi))
