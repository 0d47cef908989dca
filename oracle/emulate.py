"""Reduced-precision emulation of the preconditioned GCR(k) solve.

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the library.  It shares
no code with the CUDA path; it builds on the FP64 oracle (sw_oracle.c) for the
operator L (Eq. 10), the lagged part P^M and the zonal rows of T (Eq. 13).

The paper measures what precision costs by emulation (Sec. 3.4): the
arithmetic runs in double precision and every stored value is rounded to a
shorter significand.  Here the same idea is applied to the storage plan of the
library's mixed-precision solve (Sec. 4.3 keeps half precision in the
preconditioner, higher precision at the poles and in the residual update):

  field                                   stored as
  r, p_l, L(p_l), L(e)                    FP32
  preconditioner stages q_mu and e        FP16 (or BF16) after division by a
                                          power-of-two row scale; FP32 on the
                                          pole-band rows
  coefficients of L and of T              FP32 (used by P^-1 and L(e))
  Phi, inner products, alpha, beta,       FP64
  true residual L(Phi) - R

The row scale is not in the paper: an IEEE half has 5 exponent bits where the
paper's emulated half keeps 11 (Sec. 4.1), so each 16-bit row is stored as
value / 2^e with 2^e the power of two just above the row's largest magnitude.

What the emulation does not reproduce: the rounding of the FP32 arithmetic
inside the stencil and the tridiagonal solve, and the order of the sums.  It
gives the expected iteration count and error of the storage plan; the mixed
result itself has no bit pattern to match (parity unpinned).
"""
from __future__ import annotations

import numpy as np

from .oracle import COEFF_KEYS, Opts, Problem, cyclic_solve

# (fraction bits, smallest normal exponent) of the IEEE formats; emin None
# means an unbounded exponent (the paper's emulated formats, Sec. 3.4)
FORMATS = {
    "fp64": None,
    "fp32": (23, -126),
    "fp16": (10, -14),
    "bf16": (7, -126),
}


def round_fmt(x, p: int, emin: int | None = None):
    """Round to p fraction bits, to nearest with ties to even.  Below 2^emin
    the spacing stays 2^(emin - p) (gradual underflow of the IEEE formats);
    emin None keeps the exponent unbounded.  Overflow is not modelled: callers
    keep magnitudes in range (the row scale bounds 16-bit values by 1)."""
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
    lead = e - 1                             # exponent of the leading bit
    if emin is not None:
        lead = np.maximum(lead, emin)
    q = lead - p                             # exponent of the last kept bit
    out = np.ldexp(np.rint(np.ldexp(x, -q)), q)
    return np.where(x == 0.0, x, out)


def store(x, fmt: str):
    """x as a field of format fmt holds it."""
    f = FORMATS[fmt]
    return np.array(x, dtype=np.float64) if f is None else round_fmt(x, *f)


def row_scale(row) -> float:
    """Power of two 2^e with max|row| in [2^(e-1), 2^e); 1 for a zero row."""
    m = float(np.max(np.abs(row)))
    if m == 0.0:
        return 1.0
    _, e = np.frexp(m)
    return float(np.ldexp(1.0, int(e)))


def store_q(q, fmt: str, band: int):
    """A preconditioner field as the mixed path stores it: rows within band of
    a pole in FP32, the others in fmt after division by their row scale."""
    q = np.array(q, dtype=np.float64)
    if FORMATS[fmt] is None:
        return q
    ny = q.shape[0]
    out = np.empty_like(q)
    for j in range(ny):
        if j < band or j >= ny - band:
            out[j] = store(q[j], "fp32")
        else:
            s = row_scale(q[j])
            out[j] = store(q[j] / s, fmt) * s
    return out


def default_band(ny: int) -> int:
    """Pole-band rows at each pole: 1/2/3 at 64/128/256 rows (Sec. 4.3), a band
    of fixed angular width in general, round(3 ny / 256) rows."""
    b = max(1, (3 * ny + 128) // 256)
    return min(b, ny // 2)


class MixedSolve:
    """GCR(k) with option-3 preconditioning (Sec. 2.3, Eq. 13) under the
    storage plan above.  The steps are those of the FP64 oracle's swo_gcr;
    every store is followed by the rounding of its field."""

    def __init__(self, coeffs: dict, qfmt: str = "fp16", vfmt: str = "fp32",
                 cfmt: str = "fp32", band: int | None = None):
        self.exact = Problem(coeffs)                     # FP64: true residual
        self.work = Problem({k: store(coeffs[k], cfmt) for k in COEFF_KEYS})
        self.qfmt, self.vfmt = qfmt, vfmt
        ny = self.exact.ny
        self.band = default_band(ny) if band is None else min(band, ny // 2)

    def precond(self, r, opts: Opts, eta: float):
        """Option 3: q_0 = 0, q_{mu+1} = T^-1 (q_mu + eta (P^M q_mu - r)), each
        stage stored in the 16-bit format."""
        W = self.work
        q = np.zeros_like(r)
        for _ in range(opts.n_rich):
            d = q + eta * (W.apply_PM(q) - r)
            q = np.empty_like(r)
            for j in range(W.ny):
                q[j] = cyclic_solve(*W.row_T(j, eta), d[j])
            q = store_q(q, self.qfmt, self.band)
        return q

    def solve(self, R, opts: Opts, phi0=None, eta: float | None = None):
        """Returns (phi, stats).  Convergence is judged on the FP64 true
        residual, recomputed from Phi when the recursive one meets the
        tolerance (the reliable update of Sec. 4)."""
        assert opts.pc == 3, "the emulation covers preconditioner option 3"
        E, W, vf = self.exact, self.work, self.vfmt
        R = np.asarray(R, dtype=np.float64)
        phi = np.zeros_like(R) if phi0 is None else np.array(phi0, dtype=np.float64)
        eta = E.eta_auto() if eta is None else eta
        k, tol = opts.k, opts.tol
        nR = float(np.sqrt(np.sum(R * R)))
        st = {"iterations": 0, "converged": 0, "true_rel_residual": 0.0, "R_norm": nR}
        if nR == 0.0:
            st["converged"] = 1
            return np.zeros_like(R), st
        rt = E.operator(phi) - R                          # step 1, FP64
        rn = float(np.sqrt(np.sum(rt * rt)))
        st["true_rel_residual"] = rn / nR
        if rn <= tol * nR and opts.min_iters <= 0:
            st["converged"] = 1
            return phi, st
        r = store(rt, vf)
        p = [self.precond(r, opts, eta)]
        Lp = [store(W.operator(p[0]), vf)]
        it = nu = 0
        while True:
            # step 2: beta minimises ||r + beta L p_nu||
            beta = -np.sum(r * Lp[nu]) / np.sum(Lp[nu] * Lp[nu])
            phi = phi + beta * p[nu]
            r = store(r + beta * Lp[nu], vf)
            it += 1
            rn = float(np.sqrt(np.sum(r * r)))
            if (rn <= tol * nR and it >= opts.min_iters) or it >= opts.max_iters or \
               (opts.ru_every > 0 and it % opts.ru_every == 0):
                rt = E.operator(phi) - R
                rn = float(np.sqrt(np.sum(rt * rt)))
                st["true_rel_residual"] = rn / nR
                if rn <= tol * nR and it >= opts.min_iters:
                    st["converged"] = 1
                    break
                if it >= opts.max_iters:
                    break
                r = store(rt, vf)
            # step 3: preconditioned residual and its image under L
            e = self.precond(r, opts, eta)
            Le = store(W.operator(e), vf)
            # step 4: orthogonalise against the cycle's directions
            alpha = [-np.sum(Le * Lp[l]) / np.sum(Lp[l] * Lp[l]) for l in range(nu + 1)]
            pn, Lpn = e.copy(), Le.copy()
            for l in range(nu + 1):
                pn += alpha[l] * p[l]
                Lpn += alpha[l] * Lp[l]
            p.append(store(pn, vf))
            Lp.append(store(Lpn, vf))
            nu += 1
            if nu == k:                                   # restart keeps p_k
                p, Lp, nu = [p[k]], [Lp[k]], 0
        st["iterations"] = it
        return phi, st


# ---------------------------------------------------------------------------
# Split fluid thickness for the residual (Sec. 4.2, Eq. 14)
# ---------------------------------------------------------------------------
# The paper computes r0 = L(Phi) - R in single precision with Phi held as two
# single-precision fields, Phi ~ Phi_hat + Phi_tilde: Phi_hat is the depth
# truncated at a refresh (every 100 steps), Phi_tilde the truncated remainder,
# to which the solver's increments are added.  In Eq. 14 the derivatives of
# Phi_hat are computed once per refresh and stored; those of Phi_tilde, their
# sums, the B and C terms on Phi_SP = Phi_hat + Phi_tilde and the divergence
# run in single precision.
#
# operator_np evaluates the flux form of L (the oracle's stencil, Eq. 10) in
# the arithmetic of `dtype` with numpy, whose float32 operations are IEEE
# single precision with rounding to nearest (one rounding per operation, no
# fused multiply-add).  With `hat` given, x is Phi_tilde and the derivative
# parts of Phi_hat come from face_gradients(hat).

def _ghost(x, dj):
    """Rows j + dj for every row j: beyond a pole, the pole row shifted by half
    a circle (the across-pole continuation of the stencil)."""
    ny, nx = x.shape
    out = np.empty_like(x)
    for j in range(ny):
        jj = j + dj
        if jj < 0:
            out[j] = np.roll(x[0], -(nx // 2))
        elif jj >= ny:
            out[j] = np.roll(x[ny - 1], -(nx // 2))
        else:
            out[j] = x[jj]
    return out


def face_gradients(x, dtype=np.float64):
    """The four derivative parts of the face fluxes of x, in dtype:
    gxl = d/dlam and gxp = d/dphi on the zonal faces (i+1/2, j), gyp = d/dphi
    and gyl = d/dlam on the meridional faces (i, j+1/2)."""
    x = np.asarray(x, dtype=dtype)
    ny, nx = x.shape
    dlam, dphi = dtype(2.0 * np.pi / nx), dtype(np.pi / ny)
    e = np.roll(x, -1, axis=1)                       # x[i+1, j]
    n, s = _ghost(x, 1), _ghost(x, -1)               # x[i, j+1], x[i, j-1]
    gxl = (e - x) / dlam
    gxp = ((n + np.roll(n, -1, axis=1)) - (s + np.roll(s, -1, axis=1))) / (dtype(4.0) * dphi)
    gyp = (n - x) / dphi
    gyl = ((e + np.roll(n, -1, axis=1)) - (np.roll(x, 1, axis=1) + np.roll(n, 1, axis=1))) / (dtype(4.0) * dlam)
    return gxl, gxp, gyp, gyl


def operator_np(coeffs: dict, x, dtype=np.float64, hat=None, hat_grads=None):
    """L(x) of Eq. 10 in dtype arithmetic; with hat (and its stored gradients
    hat_grads), L(hat + x) by Eq. 14: derivatives as stored ones of hat plus
    those of x, the B and C terms on the dtype sum hat + x."""
    x = np.asarray(x, dtype=dtype)
    ny, nx = x.shape
    dlam, dphi = dtype(2.0 * np.pi / nx), dtype(np.pi / ny)
    half = dtype(0.5)

    def xmean(c):                                    # face means, rounded to dtype
        return (0.5 * (c + np.roll(c, -1, axis=1))).astype(dtype)

    def ymean(c):
        m = np.zeros_like(c)
        m[:-1] = 0.5 * (c[:-1] + c[1:])
        return m.astype(dtype)

    a11, a12, b1 = (xmean(coeffs[k]) for k in ("A11", "A12", "B1"))
    a22, a21, b2 = (ymean(coeffs[k]) for k in ("A22", "A21", "B2"))
    C = np.asarray(coeffs["C"]).astype(dtype)
    gxl, gxp, gyp, gyl = face_gradients(x, dtype)
    sp = x
    if hat is not None:
        h = [np.asarray(g).astype(dtype) for g in hat_grads]
        gxl, gxp, gyp, gyl = gxl + h[0], gxp + h[1], gyp + h[2], gyl + h[3]
        sp = np.asarray(hat, dtype=dtype) + x
    fx = a11 * gxl + a12 * gxp + b1 * (half * (sp + np.roll(sp, -1, axis=1)))
    fy = a22 * gyp + a21 * gyl + b2 * (half * (sp + _ghost(sp, 1)))
    fy[-1] = 0                                       # no flux through the pole faces
    fys = np.zeros_like(fy)
    fys[1:] = fy[:-1]
    return (fx - np.roll(fx, 1, axis=1)) / dlam + (fy - fys) / dphi - C * sp


def split_phi(phi):
    """(Phi_hat, Phi_tilde) of a refresh: Phi_hat = fp32(Phi), Phi_tilde =
    fp32(Phi - Phi_hat) with the difference taken in double precision."""
    phi = np.asarray(phi, dtype=np.float64)
    hat = phi.astype(np.float32)
    return hat, (phi - hat.astype(np.float64)).astype(np.float32)
