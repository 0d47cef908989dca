"""The split fluid thickness of Sec. 4.2, Eq. 14 on the GPU (sw_split_refresh,
sw_split_residual, and split_r0 in the solver) against the emulation oracle
(oracle/emulate.py: operator_np with hat and hat_grads).

- Element-wise: the GPU's single-precision r0 and the emulation's differ by
  at most 16 units of FP32 rounding of the terms they sum (both evaluate the
  same flux form in FP32; they round in other places: the emulation divides
  by the grid spacings, the library folds them into the face coefficients).
- The point of Eq. 14: near the poles the split r0 is orders of magnitude
  closer to the FP64 residual than r0 from Phi truncated to FP32.
- In the solver: a mixed solve whose first residual comes from the split form
  reaches the FP64 true residual and the oracle's solution.
"""
import numpy as np
import pytest

import oracle as O
from oracle import emulate as E
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16120_gb300 as sw  # noqa: E402

U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2103_16120_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def full_depth_case(nx, ny, seed):
    """Coefficients of a synthetic state, its full depth Phi* (about 8000 m) as
    the current Phi, and R one solver increment away (as in the emulation's
    own pins of Eq. 14)."""
    st = synth.synthetic_state(nx, ny, seed)
    P = synth.coefficients(st)
    P["R"] = synth.rhs_divergence(nx, ny, seed)
    dphi, _ = O.Problem(P).gcr(P["R"], O.Opts(tol=1e-12, max_iters=4000))
    phin = st.phi_star.copy()
    P["R"] = O.Problem(P).operator(phin + dphi)
    return P, phin


def term_scale(P, x):
    """Per point, the sum of the magnitudes of the terms the flux form of
    Eq. 10 adds up for x: the scale of FP32 rounding in any evaluation."""
    ny, nx = x.shape
    dlam, dphi = 2 * np.pi / nx, np.pi / ny
    e = np.roll(x, -1, axis=1)
    n, s = E._ghost(x, 1), E._ghost(x, -1)
    xm = lambda c: 0.5 * (c + np.roll(c, -1, axis=1))          # noqa: E731
    def ym(c):
        m = np.zeros_like(c); m[:-1] = 0.5 * (c[:-1] + c[1:]); return m
    fx = (np.abs(xm(P["A11"])) * np.abs(e - x) / dlam
          + np.abs(xm(P["A12"])) * (np.abs(n) + np.abs(np.roll(n, -1, axis=1)) + np.abs(s)
                                    + np.abs(np.roll(s, -1, axis=1))) / (4 * dphi)
          + np.abs(xm(P["B1"])) * 0.5 * (np.abs(x) + np.abs(e)))
    fy = (np.abs(ym(P["A22"])) * np.abs(n - x) / dphi
          + np.abs(ym(P["A21"])) * (np.abs(e) + np.abs(np.roll(n, -1, axis=1)) + np.abs(np.roll(x, 1, axis=1))
                                    + np.abs(np.roll(n, 1, axis=1))) / (4 * dlam)
          + np.abs(ym(P["B2"])) * 0.5 * (np.abs(x) + np.abs(n)))
    fy[-1] = 0
    fys = np.zeros_like(fy); fys[1:] = fy[:-1]
    return (fx + np.roll(fx, 1, axis=1)) / dlam + (fy + fys) / dphi + np.abs(P["C"] * x)


def gpu_grid(P):
    ny, nx = P["C"].shape
    g = sw.sw_grid_create(nx, ny)
    sw.sw_elliptic_set_coeffs(g, *[dev(P[k]) for k in sw.COEFF_KEYS])
    return g


@pytest.mark.parametrize("nx,ny", [(256, 128), (512, 256), (136, 40)])
def test_split_residual_matches_the_emulation(nx, ny):
    P, phin = full_depth_case(nx, ny, 25 + nx)
    g = gpu_grid(P)
    phi_d, R_d = dev(phin), dev(P["R"])
    sw.sw_split_refresh(g, phi_d)
    r = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
    sw.sw_split_residual(g, phi_d, R_d, r)
    hat, tilde = E.split_phi(phin)
    hg = [q.astype(np.float32) for q in E.face_gradients(hat.astype(np.float64))]
    emu = E.operator_np(P, tilde, np.float32, hat=hat, hat_grads=hg).astype(np.float64) - P["R"]
    got = r.cpu().numpy().astype(np.float64)
    S = term_scale(P, phin) + np.abs(P["R"])
    bad = np.abs(got - emu) > 16 * U32 * S
    assert not bad.any(), f"{bad.sum()} points, worst {np.max(np.abs(got - emu) / (U32 * S)):.1f} ulps of the terms"


def test_split_residual_recovers_the_pole_rows():
    """Sec. 4.2: near the poles, r0 from the split thickness is far closer to
    the FP64 residual than r0 from Phi truncated to FP32.  (Away from the poles
    the full operator's FP32 error is set by the rounding of C Phi and R, which
    the split does not touch.)  The GPU's split r0 is as close to the FP64
    residual as the emulation's."""
    nx, ny = 256, 128
    P, phin = full_depth_case(nx, ny, 31)
    g = gpu_grid(P)
    phi_d, R_d = dev(phin), dev(P["R"])
    sw.sw_split_refresh(g, phi_d)
    r = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
    sw.sw_split_residual(g, phi_d, R_d, r)
    exact = O.Problem(P).operator(phin) - P["R"]
    y32 = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
    sw.sw_operator_apply(g, dev(phin, torch.float32), y32)          # Phi truncated to FP32, FP32 operator
    plain = y32.cpu().numpy().astype(np.float64) - P["R"]

    def rowerr(x):
        return np.sqrt(np.sum((x - exact) ** 2, axis=1)) / np.sqrt(np.sum(exact ** 2, axis=1))

    es, ep = rowerr(r.cpu().numpy().astype(np.float64)), rowerr(plain)
    assert max(ep[0], ep[-1]) >= 100 * max(es[0], es[-1])
    hat, tilde = E.split_phi(phin)
    hg = [q.astype(np.float32) for q in E.face_gradients(hat.astype(np.float64))]
    ee = rowerr(E.operator_np(P, tilde, np.float32, hat=hat, hat_grads=hg).astype(np.float64) - P["R"])
    assert np.median(es) <= 2 * np.median(ee) and max(es[0], es[-1]) <= 2 * max(ee[0], ee[-1])


@pytest.mark.parametrize("row_mode", [1, 2])
@pytest.mark.parametrize("prec", [sw.SW_PREC_MIXED_FP16, sw.SW_PREC_MIXED_BF16])
def test_solver_with_split_initial_residual(prec, row_mode):
    nx, ny = 256, 128
    P, phin = full_depth_case(nx, ny, 41)
    g = gpu_grid(P)
    R_d = dev(P["R"])
    out = {}
    for split in (0, 1):
        phi = dev(phin)
        if split:
            sw.sw_split_refresh(g, phi)
        o = sw.sw_solve_opts_default(prec=prec, tol=1e-8, max_iters=2000, row_mode=row_mode, split_r0=split)
        st = sw.sw_gcr_solve(g, o, R_d, phi)
        assert st.status == sw.SW_OK and st.true_rel_residual <= 1e-8, st.as_dict()
        out[split] = (st, phi.cpu().numpy())
    ref, _ = O.Problem(P).gcr(P["R"], O.Opts(tol=1e-12, max_iters=4000), phi0=phin)
    x = out[1][1]
    assert np.linalg.norm(O.Problem(P).operator(x) - P["R"]) <= 1e-8 * np.linalg.norm(P["R"]) * (1 + 1e-9)
    assert np.linalg.norm(x - ref) <= 1e-6 * np.linalg.norm(ref)
    # the initial residual norm agrees with the FP64 one to FP32 accuracy
    assert abs(out[1][0].r0_norm - out[0][0].r0_norm) <= 1e-4 * out[0][0].r0_norm
    assert out[1][0].iterations <= out[0][0].iterations + 4


def test_split_argument_checks():
    P, phin = full_depth_case(64, 32, 51)
    g = gpu_grid(P)
    R_d, phi = dev(P["R"]), dev(phin)
    o = sw.sw_solve_opts_default(prec=sw.SW_PREC_MIXED_FP16, split_r0=1)
    with pytest.raises(sw.SwError) as ei:          # no refresh yet
        sw.sw_gcr_solve(g, o, R_d, phi.clone())
    assert ei.value.status == sw.SW_ERR_INVALID_ARG
    with pytest.raises(sw.SwError):
        sw.sw_split_residual(g, phi, R_d, torch.empty((32, 64), dtype=torch.float32, device="cuda"))
    sw.sw_split_refresh(g, phi)
    with pytest.raises(sw.SwError):                # FP64 keeps the FP64 initial residual
        sw.sw_gcr_solve(g, sw.sw_solve_opts_default(split_r0=1), R_d, phi.clone())
    g2 = sw.sw_grid_create(68, 16)                 # nx not a multiple of 8
    with pytest.raises(sw.SwError):
        sw.sw_split_refresh(g2, torch.zeros((16, 68), dtype=torch.float64, device="cuda"))
