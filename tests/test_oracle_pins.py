"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own formulas: closed forms,
the continuous operator of Eq. 10 (differentiated symbolically), invariants,
dense brute-force solves and the numbers the paper prints.  Together they are
chosen so that a dropped term, a wrong sign or index, or a transposed operand
anywhere in the oracle fails one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import synth
from synth.sphere import grid_coords, real_sh

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _const_coeffs(nx, ny, **vals):
    z = np.zeros((ny, nx))
    out = {k: z.copy() for k in O.COEFF_KEYS}
    for k, v in vals.items():
        out[k] = np.broadcast_to(v, (ny, nx)).astype(np.float64).copy()
    return out


# --------------------------------------------------------------------------
# the generator's spherical harmonics (used by the eigenfunction pin)
# --------------------------------------------------------------------------
def test_real_sh_orthonormal_and_matches_scipy():
    sp = pytest.importorskip("scipy.special")
    lam, phi, dlam, dphi = grid_coords(64, 32)
    for (l, m) in [(1, 0), (2, 1), (4, -3), (8, 4)]:
        y = real_sh(l, m, lam, phi)
        if hasattr(sp, "sph_harm_y"):
            th = (0.5 * np.pi - phi)[:, None] + 0 * lam[None, :]
            ph = lam[None, :] + 0 * phi[:, None]
            z = sp.sph_harm_y(l, abs(m), th, ph)
        else:
            th = (0.5 * np.pi - phi)[:, None] + 0 * lam[None, :]
            ph = lam[None, :] + 0 * phi[:, None]
            z = sp.sph_harm(abs(m), l, ph, th)
        ref = z.real if m >= 0 else z.imag
        if m != 0:
            ref = math.sqrt(2.0) * ref
        # scipy includes the Condon-Shortley phase (-1)^m
        ref = ref * (-1) ** abs(m)
        assert np.allclose(y, ref, atol=1e-12)
    # orthonormality on a fine grid (midpoint rule in phi, exact in lambda)
    lam, phi, dlam, dphi = grid_coords(128, 256)
    w = np.cos(phi)[:, None] * dlam * dphi
    a = real_sh(3, 2, lam, phi)
    b = real_sh(5, 2, lam, phi)
    assert abs(np.sum(w * a * a) - 1) < 1e-3
    assert abs(np.sum(w * a * b)) < 1e-6


# --------------------------------------------------------------------------
# operator L (Eq. 10)
# --------------------------------------------------------------------------
def test_op_closed_form_zonal_fourier_mode():
    """A11 = const, C = const, Phi = cos(m lambda): the three-point zonal
    difference has the exact eigenvalue -(A11 (2 - 2 cos m dlam)/dlam^2 + C)."""
    nx, ny = 48, 6
    a0, c0 = 3.7e7, 2.1e9
    prob = O.Problem(_const_coeffs(nx, ny, A11=a0, C=c0))
    lam, phi, dlam, dphi = grid_coords(nx, ny)
    for m in (1, 5, 24):
        x = np.broadcast_to(np.cos(m * lam), (ny, nx)).copy()
        y = prob.operator(x)
        lamb = -(a0 * (2 - 2 * math.cos(m * dlam)) / dlam ** 2 + c0)
        assert np.max(np.abs(y - lamb * x)) <= 1e-14 * abs(lamb)


def test_op_closed_form_B_terms():
    """B1 = const: L x = B1 (x[i+1] - x[i-1])/(2 dlam) exactly; for x = sin(lambda)
    that is B1 cos(lambda) sin(dlam)/dlam.  B2 = const with x = sin(phi): interior
    rows give B2 cos(phi) sin(dphi)/dphi exactly."""
    nx, ny = 32, 16
    lam, phi, dlam, dphi = grid_coords(nx, ny)
    prob = O.Problem(_const_coeffs(nx, ny, B1=2.5))
    x = np.broadcast_to(np.sin(lam), (ny, nx)).copy()
    y = prob.operator(x)
    assert np.allclose(y, 2.5 * np.cos(lam)[None, :] * math.sin(dlam) / dlam, atol=1e-13)
    prob = O.Problem(_const_coeffs(nx, ny, B2=-1.5))
    x = np.broadcast_to(np.sin(phi)[:, None], (ny, nx)).copy()
    y = prob.operator(x)
    exp = -1.5 * np.cos(phi)[:, None] * math.sin(dphi) / dphi
    assert np.allclose(y[1:-1], np.broadcast_to(exp, (ny, nx))[1:-1], atol=1e-13)
    # pole rows: only the inner face carries flux, B2 (x_0 + x_1)/2 / dphi
    assert np.allclose(y[0], -1.5 * 0.5 * (x[0] + x[1]) / dphi, atol=1e-13)
    assert np.allclose(y[-1], 1.5 * 0.5 * (x[-2] + x[-1]) / dphi, atol=1e-13)


def test_op_closed_form_cross_terms_interior():
    """A12 = const (or A21 = const), x = sin(lambda) sin(phi): on interior rows
    both cross terms reduce to A cos(lambda) cos(phi) sin(dlam) sin(dphi)/(dlam dphi)."""
    nx, ny = 32, 16
    lam, phi, dlam, dphi = grid_coords(nx, ny)
    x = np.sin(lam)[None, :] * np.sin(phi)[:, None]
    exp = np.cos(lam)[None, :] * np.cos(phi)[:, None] * math.sin(dlam) * math.sin(dphi) / (dlam * dphi)
    for key in ("A12", "A21"):
        prob = O.Problem(_const_coeffs(nx, ny, **{key: 0.8}))
        y = prob.operator(x)
        assert np.allclose(y[1:-1], 0.8 * exp[1:-1], atol=1e-13)


def _sym_operator(nx, ny):
    """Smooth coefficient fields (polynomials in the Cartesian coordinates of
    the unit sphere; A22, A21, B2 carry cos(phi) so the meridional flux vanishes
    at the poles as in the model), a smooth Phi, and the continuous
    L(Phi) = d/dlam(A11 Phi_lam + A12 Phi_phi + B1 Phi)
           + d/dphi(A21 Phi_lam + A22 Phi_phi + B2 Phi) - C Phi   (Eq. 10)."""
    sp = pytest.importorskip("sympy")
    L, F = sp.symbols("lam phi", real=True)
    X, Y, Z = sp.cos(F) * sp.cos(L), sp.cos(F) * sp.sin(L), sp.sin(F)
    co = {
        "A11": 1 + sp.Rational(3, 10) * X + sp.Rational(1, 5) * Z ** 2,
        "A12": sp.Rational(1, 2) * (1 + X * Z),
        "A21": sp.Rational(1, 2) * sp.cos(F) * (Z + sp.Rational(3, 10) * X),
        "A22": sp.cos(F) * (1 + sp.Rational(1, 5) * Y),
        "B1": sp.Rational(3, 10) * (X + sp.Rational(1, 2) * Y * Z),
        "B2": sp.Rational(2, 5) * sp.cos(F) * (Y - Z),
        "C": 2 + Z,
    }
    Phi = X * Z + Y ** 2 + sp.Rational(1, 2) * Z ** 3 + X
    Lc = (sp.diff(co["A11"] * sp.diff(Phi, L) + co["A12"] * sp.diff(Phi, F) + co["B1"] * Phi, L)
          + sp.diff(co["A21"] * sp.diff(Phi, L) + co["A22"] * sp.diff(Phi, F) + co["B2"] * Phi, F)
          - co["C"] * Phi)
    lam, phi, _, _ = grid_coords(nx, ny)
    LL, FF = np.meshgrid(lam, phi)
    ev = lambda e: np.broadcast_to(sp.lambdify((L, F), e, "numpy")(LL, FF), (ny, nx)).astype(float).copy()
    return {k: ev(v) for k, v in co.items()}, ev(Phi), ev(Lc)


def test_op_converges_to_continuous_operator():
    """Every term, sign and index of the discrete operator: the discrete L
    applied to a smooth field converges to the symbolic continuous operator,
    at second order on interior rows and at first order on the two pole rows,
    where the exact zero pole-face flux meets the O(h^2) inner-face flux
    (divided by dphi).  A wrong across-pole continuation or a dropped term
    leaves an O(1) error that does not converge at all."""
    errs_in, errs_pole = [], []
    for nx, ny in [(32, 16), (64, 32), (128, 64), (256, 128)]:
        co, phi, Lc = _sym_operator(nx, ny)
        y = O.Problem(co).operator(phi)
        d = np.abs(y - Lc)
        errs_in.append(d[1:-1].max())
        errs_pole.append(max(d[0].max(), d[-1].max()))
    r_in = [errs_in[i] / errs_in[i + 1] for i in range(3)]
    r_pole = [errs_pole[i] / errs_pole[i + 1] for i in range(3)]
    assert min(r_in) > 3.5, (errs_in, r_in)
    assert min(r_pole) > 1.8 and errs_pole[-1] < 0.05 * errs_pole[0], (errs_pole, r_pole)


@pytest.mark.parametrize("lm", [(1, 0), (2, 1), (4, 3), (8, 4)])
def test_op_sh_eigenfunctions_second_order(lm):
    """Constant-coefficient reduction A11 = k/cos(phi), A22 = k cos(phi), C = c0 cos(phi):
    L Y_lm = -cos(phi) (k l(l+1) + c0) Y_lm for the continuous operator; the
    discrete error (cos-weighted L2) falls by ~4 per halving of the mesh."""
    l, m = lm
    kap, c0 = 1.3, 0.7
    errs = []
    for nx, ny in [(32, 16), (64, 32), (128, 64), (256, 128)]:
        lam, phi, dlam, dphi = grid_coords(nx, ny)
        cphi = np.cos(phi)[:, None]
        co = _const_coeffs(nx, ny)
        co["A11"] = np.broadcast_to(kap / cphi, (ny, nx)).copy()
        co["A22"] = np.broadcast_to(kap * cphi, (ny, nx)).copy()
        co["C"] = np.broadcast_to(c0 * cphi, (ny, nx)).copy()
        Y = real_sh(l, m, lam, phi)
        y = O.Problem(co).operator(Y)
        exact = -cphi * (kap * l * (l + 1) + c0) * Y
        w = cphi * dlam * dphi
        errs.append(math.sqrt(np.sum(w * (y - exact) ** 2) / np.sum(w * exact ** 2)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert min(orders) >= 1.9, (errs, orders)


def test_op_zero_sum_invariant():
    """Divergence form + periodic longitude + zero pole-face flux:
    sum_ij (L x + C x) = 0 for any x and any coefficients."""
    rng = np.random.default_rng(3)
    nx, ny = 24, 12
    co = {k: rng.standard_normal((ny, nx)) for k in O.COEFF_KEYS}
    prob = O.Problem(co)
    x = rng.standard_normal((ny, nx))
    y = prob.operator(x) + co["C"] * x
    dlam, dphi = 2 * math.pi / nx, math.pi / ny
    scale = np.sum(np.abs(y)) + np.sum(np.abs(co["C"] * x))
    # the flux differences carry 1/dlam and 1/dphi: sum(y) telescopes to zero
    assert abs(np.sum(y)) <= 1e-13 * scale


def test_op_coriolis_cancellation():
    """A12 = -A21 = const (the rotational part of A): the two cross terms cancel
    exactly on rows 1..ny-2."""
    rng = np.random.default_rng(4)
    nx, ny = 20, 10
    prob = O.Problem(_const_coeffs(nx, ny, A12=1.7, A21=-1.7))
    x = rng.standard_normal((ny, nx))
    y = prob.operator(x)
    assert np.max(np.abs(y[1:-1])) <= 1e-13 * np.max(np.abs(x)) / (2 * math.pi / nx * math.pi / ny)


def test_op_symmetric_negative_definite():
    """A12 = A21 = 0, B = 0: L is self-adjoint and negative definite."""
    rng = np.random.default_rng(5)
    nx, ny = 16, 8
    co = _const_coeffs(nx, ny)
    co["A11"] = 1 + rng.random((ny, nx))
    co["A22"] = 1 + rng.random((ny, nx))
    co["C"] = 0.1 + rng.random((ny, nx))
    M = O.operator_matrix(O.Problem(co))
    assert np.max(np.abs(M - M.T)) <= 1e-13 * np.max(np.abs(M))
    assert np.max(np.linalg.eigvalsh(0.5 * (M + M.T))) < 0
    # with the Coriolis cross terms (A12 = -A21) the symmetric part is unchanged
    co["A12"] = np.full((ny, nx), 0.6)
    co["A21"] = -co["A12"]
    M2 = O.operator_matrix(O.Problem(co))
    sym2 = 0.5 * (M2 + M2.T)
    assert np.max(np.linalg.eigvalsh(sym2)) < 0


def test_physical_operator_negative_definite():
    """The synthetic problem's L (all terms) is negative definite (Sec. 2.2)."""
    P = synth.problem(16, 8, 11)
    M = O.operator_matrix(O.Problem(P))
    assert np.max(np.linalg.eigvalsh(0.5 * (M + M.T))) < 0


def test_diag_L_matches_assembled_matrix():
    P = synth.problem(16, 8, 12)
    prob = O.Problem(P)
    M = O.operator_matrix(prob)
    d = prob.diag_L().ravel()
    assert np.allclose(d, np.diag(M), rtol=1e-13, atol=0)


def test_split_PZ_closed_form_and_PM_remainder():
    """P^Z on a Fourier mode (constant A11) and P^M = L - P^Z + C by brute force:
    L = (P^Z - P^H) + P^M with P^H = C (Eq. 13)."""
    nx, ny = 16, 8
    P = synth.problem(nx, ny, 13)
    prob = O.Problem(P)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((ny, nx))
    lhs = prob.apply_PZ(x) - P["C"] * x + prob.apply_PM(x)
    assert np.allclose(lhs, prob.operator(x), rtol=0, atol=1e-12 * np.abs(prob.operator(x)).max())
    # P^Z alone, constant A11 on a Fourier mode
    lam, phi, dlam, dphi = grid_coords(nx, ny)
    probc = O.Problem(_const_coeffs(nx, ny, A11=2.0, A22=5.0, C=1.0))
    xm = np.broadcast_to(np.cos(3 * lam), (ny, nx)).copy()
    assert np.allclose(probc.apply_PZ(xm), -2.0 * (2 - 2 * math.cos(3 * dlam)) / dlam ** 2 * xm, atol=1e-12)
    # P^M carries no zonal-only second derivative: it vanishes on x = f(lambda)
    # when A22, A12, A21, B are zero
    probz = O.Problem(_const_coeffs(nx, ny, A11=2.0, C=1.0))
    assert np.max(np.abs(probz.apply_PM(xm))) < 1e-12


# --------------------------------------------------------------------------
# eta, the pseudo time step of Eq. 13 (Sec. 2.3): 1 / max |diag(P^M)|
# --------------------------------------------------------------------------
def test_eta_auto_closed_form_meridional_diffusion():
    """A22 = kappa alone: P^M is the meridional second difference with zero flux
    through the pole faces, so diag(P^M) is -2 kappa/dphi^2 on interior rows and
    -kappa/dphi^2 on the two pole rows; eta = dphi^2 / (2 kappa)."""
    for nx, ny, kappa in [(16, 8, 3.5e6), (48, 20, 0.7), (8, 3, 1e12)]:
        _, _, _, dphi = grid_coords(nx, ny)
        eta = O.Problem(_const_coeffs(nx, ny, A22=kappa)).eta_auto()
        assert abs(eta - dphi ** 2 / (2 * kappa)) <= 1e-14 * eta
    # two rows: both are pole rows, each with one meridional face
    _, _, _, dphi = grid_coords(8, 2)
    eta = O.Problem(_const_coeffs(8, 2, A22=2.0)).eta_auto()
    assert abs(eta - dphi ** 2 / 2.0) <= 1e-14 * eta


def test_eta_auto_ignores_the_implicit_part_and_the_cross_terms():
    """The zonal A11 part and C form T = I - eta (P^Z - P^H) and are not in P^M;
    the cross terms A12, A21 never touch the centre point (even across a pole,
    where the ghost is shifted by nx/2).  Adding any of them leaves eta at the
    closed form of A22 alone.  Fails for diag(L) in place of diag(P^M), a
    dropped +C or a dropped A11 removal."""
    nx, ny, kappa = 24, 12, 4.0e5
    _, _, _, dphi = grid_coords(nx, ny)
    rng = np.random.default_rng(31)
    c = _const_coeffs(nx, ny, A22=kappa)
    c["A11"] = 1e7 * (1 + rng.random((ny, nx)))
    c["C"] = 1e9 * (1 + rng.random((ny, nx)))
    c["A12"] = 3e5 * rng.standard_normal((ny, nx))
    c["A21"] = -c["A12"] + 1e5 * rng.standard_normal((ny, nx))
    eta = O.Problem(c).eta_auto()
    assert abs(eta - dphi ** 2 / (2 * kappa)) <= 1e-13 * eta


def test_eta_auto_closed_form_advective_terms():
    """B2 = b (constant) with A22 = kappa: the centred meridional mean puts
    +b/(2 dphi) on the first row (north face only) and -b/(2 dphi) on the last
    (south face only), and cancels inside.  With b > 2 kappa/dphi the pole rows
    set eta = 1 / (kappa/dphi^2 + b/(2 dphi)).  B1 = beta sin(lambda) alone puts
    (B1[i+1] - B1[i-1]) / (4 dlam) = beta cos(lambda_i) sin(dlam) / (2 dlam) on
    the diagonal, largest at lambda = 0: eta = 2 dlam / (beta sin dlam).  A
    dropped or mis-signed B term fails these."""
    nx, ny, kappa = 32, 16, 1.0
    lam, _, dlam, dphi = grid_coords(nx, ny)
    b = 5 * kappa / dphi
    eta = O.Problem(_const_coeffs(nx, ny, A22=kappa, B2=b)).eta_auto()
    want = 1.0 / (kappa / dphi ** 2 + b / (2 * dphi))
    assert abs(eta - want) <= 1e-14 * want
    # B2 alone: only the pole rows see it
    eta = O.Problem(_const_coeffs(nx, ny, B2=b)).eta_auto()
    assert abs(eta - 2 * dphi / b) <= 1e-14 * eta
    beta = 7.0
    eta = O.Problem(_const_coeffs(nx, ny, B1=beta * np.sin(lam)[None, :])).eta_auto()
    want = 2 * dlam / (beta * math.sin(dlam))
    assert abs(eta - want) <= 1e-13 * want


def test_eta_auto_equals_assembled_PM_diagonal():
    """Brute force on the synthetic problem: assemble P^M column by column
    (P^M = L - P^Z + C, itself pinned above) and take 1/max|diag|."""
    nx, ny = 16, 8
    P = synth.problem(nx, ny, 17)
    prob = O.Problem(P)
    n = nx * ny
    dm = np.empty(n)
    for c in range(n):
        e = np.zeros(n); e[c] = 1.0
        dm[c] = prob.apply_PM(e.reshape(ny, nx)).ravel()[c]
    assert abs(prob.eta_auto() - 1.0 / np.max(np.abs(dm))) <= 1e-13 / np.max(np.abs(dm))


# --------------------------------------------------------------------------
# cyclic tridiagonal solve and the preconditioner (Eq. 13)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [3, 4, 7, 64, 129])
def test_cyclic_solve_matches_dense(n):
    rng = np.random.default_rng(n)
    sub = -rng.random(n)
    sup = -rng.random(n)
    diag = 2.5 + rng.random(n)
    rhs = rng.standard_normal(n)
    T = np.zeros((n, n))
    for i in range(n):
        T[i, i] = diag[i]
        T[i, (i - 1) % n] += sub[i]
        T[i, (i + 1) % n] += sup[i]
    x = O.cyclic_solve(sub, diag, sup, rhs)
    ref = np.linalg.solve(T, rhs)
    assert np.max(np.abs(x - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_row_T_and_solve_fourier_closed_form():
    """Constant row coefficients: T = I - eta (P^Z - P^H) is circulant and
    T^{-1} cos(m lambda) = cos(m lambda) / (1 + eta (A11 (2 - 2 cos m dlam)/dlam^2 + C))."""
    nx, ny = 32, 4
    a0, c0, eta = 3.0, 0.5, 0.37
    prob = O.Problem(_const_coeffs(nx, ny, A11=a0, C=c0))
    lam, _, dlam, _ = grid_coords(nx, ny)
    sub, diag, sup = prob.row_T(1, eta)
    for m in (0, 1, 7, 16):
        rhs = np.cos(m * lam)
        q = O.cyclic_solve(sub, diag, sup, rhs)
        t = 1 + eta * (a0 * (2 - 2 * math.cos(m * dlam)) / dlam ** 2 + c0)
        assert np.allclose(q, rhs / t, atol=1e-14)


def test_precond_option3_two_sweeps_closed_form():
    """With P^M = 0 two Richardson sweeps give q1 = T^{-1}(-eta r),
    q2 = T^{-1}(q1 - eta r): for r = cos(m lambda), q2 = -eta r (1/t + 1/t^2)."""
    nx, ny = 32, 6
    a0, c0, eta = 3.0, 0.5, 0.21
    prob = O.Problem(_const_coeffs(nx, ny, A11=a0, C=c0))
    lam, _, dlam, _ = grid_coords(nx, ny)
    m = 5
    r = np.broadcast_to(np.cos(m * lam), (ny, nx)).copy()
    t = 1 + eta * (a0 * (2 - 2 * math.cos(m * dlam)) / dlam ** 2 + c0)
    q = prob.precond(r, O.Opts(pc=3, n_rich=2), eta=eta)
    assert np.allclose(q, -eta * r * (1 / t + 1 / t ** 2), atol=1e-14)
    q1 = prob.precond(r, O.Opts(pc=3, n_rich=1), eta=eta)
    assert np.allclose(q1, -eta * r / t, atol=1e-14)


def test_precond_option3_converges_to_inverse():
    """Many semi-implicit Richardson iterations converge to L^{-1} r (dense
    brute force): the split P^Z - P^H + P^M reassembles L."""
    P = synth.problem(16, 8, 14)
    prob = O.Problem(P)
    M = O.operator_matrix(prob)
    r = np.random.default_rng(7).standard_normal((8, 16))
    ref = np.linalg.solve(M, r.ravel()).reshape(8, 16)
    q = prob.precond(r, O.Opts(pc=3, n_rich=400))
    assert np.linalg.norm(q - ref) <= 1e-10 * np.linalg.norm(ref)


def test_precond_options_0_1_2_brute_force():
    P = synth.problem(16, 8, 15)
    prob = O.Problem(P)
    M = O.operator_matrix(prob)
    D = np.diag(M).reshape(8, 16)
    r = np.random.default_rng(8).standard_normal((8, 16))
    assert np.array_equal(prob.precond(r, O.Opts(pc=0)), r)
    assert np.allclose(prob.precond(r, O.Opts(pc=1)), r / D, rtol=1e-14, atol=0)
    q = np.zeros(r.size)
    for _ in range(3):
        q = q + 0.8 * (r.ravel() - M @ q) / D.ravel()
    assert np.allclose(prob.precond(r, O.Opts(pc=2, n_rich=3, omega=0.8)).ravel(), q, rtol=1e-12, atol=0)


# --------------------------------------------------------------------------
# GCR(k)
# --------------------------------------------------------------------------
def test_gcr_matches_dense_solve():
    P = synth.problem(16, 8, 16)
    prob = O.Problem(P)
    M = O.operator_matrix(prob)
    ref = np.linalg.solve(M, P["R"].ravel()).reshape(8, 16)
    for pc in (0, 1, 2, 3):
        phi, st = prob.gcr(P["R"], O.Opts(tol=1e-13, pc=pc, max_iters=2000))
        assert st["converged"] == 1
        assert np.linalg.norm(phi - ref) <= 1e-10 * np.linalg.norm(ref), pc


def test_gcr_without_restart_terminates_in_n_steps():
    """Unrestarted GCR is a minimal-residual Krylov method: at most n = 128
    iterations on a 16x8 grid (exact arithmetic; rounding allows a few more)."""
    P = synth.problem(16, 8, 17)
    prob = O.Problem(P)
    phi, st = prob.gcr(P["R"], O.Opts(k=200, tol=1e-12, pc=0, max_iters=400))
    assert st["converged"] == 1 and st["iterations"] <= 128 + 4


def test_gcr_minimal_residual_and_orthogonality():
    P = synth.problem(64, 32, 18)
    prob = O.Problem(P)
    phi, st, hist, orth = prob.gcr(P["R"], O.Opts(tol=1e-12, max_iters=300), want_history=True)
    assert st["converged"] == 1
    assert np.all(np.diff(hist) <= 1e-14)
    assert np.nanmax(orth) <= 1e-10


def test_gcr_recursive_equals_true_residual_fp64():
    P = synth.problem(64, 32, 19)
    prob = O.Problem(P)
    phi, st = prob.gcr(P["R"], O.Opts(tol=1e-11, max_iters=300))
    r = prob.operator(phi) - P["R"]
    nR = np.linalg.norm(P["R"])
    assert abs(st["recursive_rel_residual"] - st["true_rel_residual"]) <= 1e-12
    assert abs(np.linalg.norm(r) / nR - st["true_rel_residual"]) <= 1e-13


def test_gcr_manufactured_solution():
    P = synth.problem(32, 16, 20)
    prob = O.Problem(P)
    x = np.random.default_rng(9).standard_normal((16, 32)) * 10
    R = prob.operator(x)
    phi, st = prob.gcr(R, O.Opts(tol=1e-13, max_iters=500))
    assert np.linalg.norm(phi - x) <= 1e-9 * np.linalg.norm(x)


def test_gcr_zero_rhs_and_converged_guess():
    P = synth.problem(16, 8, 21)
    prob = O.Problem(P)
    phi, st = prob.gcr(np.zeros((8, 16)), O.Opts(), phi0=np.ones((8, 16)))
    assert st["iterations"] == 0 and np.all(phi == 0) and st["converged"] == 1
    ex, _ = prob.gcr(P["R"], O.Opts(tol=1e-13))
    phi, st = prob.gcr(P["R"], O.Opts(tol=1e-8, min_iters=0), phi0=ex)
    assert st["iterations"] == 0 and st["converged"] == 1


def test_gcr_min_iters_and_max_iters():
    P = synth.problem(32, 16, 22)
    prob = O.Problem(P)
    _, st = prob.gcr(P["R"], O.Opts(tol=1e-1, min_iters=4))
    assert st["iterations"] == 4 and st["converged"] == 1
    _, st = prob.gcr(P["R"], O.Opts(tol=0.0, max_iters=5))
    assert st["iterations"] == 5 and st["converged"] == 0 and st["status"] == 4


# --------------------------------------------------------------------------
# the paper's qualitative findings, reproduced by the oracle
# --------------------------------------------------------------------------
def test_preconditioner_option_ordering():
    """Options 1/2/3 cut GCR iterations relative to option 0 (Sec. 2.3: about
    10/40/98 percent); option 3 must cut them by at least the bulk of that."""
    red = GOLDEN["precond_iteration_reduction_percent"]["value"]
    P = synth.problem(128, 64, 23)
    prob = O.Problem(P)
    its = [prob.gcr(P["R"], O.Opts(tol=1e-10, pc=pc, max_iters=2000))[1]["iterations"] for pc in range(4)]
    assert its[0] >= its[1] >= its[2] >= its[3]
    assert its[3] <= (1 - 0.8 * red["3"] / 100) * its[0] + 1


def test_polar_absorber_helps_convergence():
    """Sec. 3.2: weak polar absorbers improve diagonal dominance; with the same
    number of iterations the final residual is not larger."""
    st = synth.synthetic_state(128, 64, 24)
    R = synth.rhs_divergence(128, 64, 24)
    res = []
    for amax in (0.0, 1.0 / (200 * 600.0)):
        prob = O.Problem(synth.coefficients(st, dt=600.0, alpha_max=amax))
        res.append(prob.gcr(R, O.Opts(tol=0.0, max_iters=4))[1]["true_rel_residual"])
    assert res[1] <= res[0] * 1.0001


def test_fp32_truncated_phi0_hurts_pole_rows_most():
    """Sec. 4.1: r0 computed from a first guess truncated to single precision
    has its largest latitude-wise relative error in the rows next to the poles."""
    P = synth.problem(256, 128, 25)
    prob = O.Problem(P)
    phi, _ = prob.gcr(P["R"], O.Opts(tol=1e-12))
    phi = phi + 8000.0   # a full fluid depth, as in the model
    R = prob.operator(phi) - prob.operator(phi - 8000.0) + P["R"]
    r_dp = prob.operator(phi) - R
    r_sp = prob.operator(phi.astype(np.float32).astype(np.float64)) - R
    num = np.sqrt(np.sum((r_sp - r_dp) ** 2, axis=1))
    den = np.sqrt(np.sum(R ** 2, axis=1))
    rel = num / den
    mid = rel[len(rel) // 4: 3 * len(rel) // 4]
    assert max(rel[0], rel[-1]) > 10 * np.median(mid)


def test_round_bits_emulates_ieee_formats():
    rng = np.random.default_rng(10)
    x = rng.standard_normal(2000) * 10.0 ** rng.uniform(-3, 3, 2000)
    assert GOLDEN["single_significand_bits"]["value"] == 23
    f32 = x.astype(np.float32).astype(np.float64)
    assert all(O.round_bits(a, 23) == b for a, b in zip(x, f32))
    f16 = x.astype(np.float16).astype(np.float64)
    p = GOLDEN["half_significand_bits"]["value"]
    ok = np.abs(x) < 6e4
    ok &= np.abs(x) > 6.2e-5
    assert all(O.round_bits(a, p) == b for a, b, m in zip(x, f16, ok) if m)
    assert abs(2.0 ** -p - GOLDEN["half_machine_epsilon"]["value"]) < 1e-6


def test_oracle_results_do_not_depend_on_the_thread_count():
    """The row loops run in parallel with fixed-order per-row partial sums, so
    one thread and all host threads give the same bits."""
    import oracle.oracle as orc
    P = synth.problem(128, 64, 5)
    outs = []
    for n in (1, 4):
        orc.set_threads(n)
        phi, st = O.Problem(P).gcr(P["R"], O.Opts(tol=1e-10, max_iters=500))
        outs.append((phi, st["iterations"]))
    orc.set_threads(os.cpu_count() or 1)
    assert outs[0][1] == outs[1][1] and np.array_equal(outs[0][0], outs[1][0])
