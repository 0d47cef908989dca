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
    """Pole-band rows at each pole: 1/2/3 at 64/128/256 rows (Sec. 4.3), one
    more per doubling of the rows."""
    b = max(1, int(np.floor(np.log2(ny))) - 5)
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
