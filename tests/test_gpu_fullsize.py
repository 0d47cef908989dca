"""Full-size checks in the launch configurations the benchmark times.

The oracle recomputes, in FP64 and with its own operator, the residual
||L(Phi) - R|| / ||R|| of the GPU's solutions:
* the 2048 x 1024 problem, mixed FP16;
* all 64 members of the 128x64 / 256x128 / 512x256 ensemble, solved in one launch;
* the first steps of the 512 x 256 warm-started sequence, whose
  solution is also compared with the oracle's own GCR solution;
* FP64 iterates on 1024 x 512 and 2048 x 1024, where every block owns several
  rows, against the oracle's iterates (1e-12);
* the largest row the library takes, 4096 x 2048, mixed FP16.

The GPU's exit test uses its FP64 true residual at tol = 1e-8.  The oracle
recomputes the same quantity in another summation order, so the bar is
1.001 * tol.
"""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16120_gb300 as sw  # noqa: E402

TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2103_16120_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def grid_for(P):
    ny, nx = P["C"].shape
    g = sw.sw_grid_create(nx, ny)
    sw.sw_elliptic_set_coeffs(g, *[torch.as_tensor(P[k], device="cuda") for k in sw.COEFF_KEYS])
    return g


def oracle_rel_residual(P, phi):
    r = O.Problem(P).operator(phi) - P["R"]
    return float(np.linalg.norm(r) / np.linalg.norm(P["R"]))


def test_large_2048x1024_mixed():
    P = synth.sequence_problem(2048, 1024, 4000, 0)
    g = grid_for(P)
    R = torch.as_tensor(P["R"], device="cuda")
    phi = torch.zeros_like(R)
    st = sw.sw_gcr_solve(g, sw.sw_solve_opts_default(prec=sw.SW_PREC_MIXED_FP16, tol=TOL, max_iters=4000), R, phi)
    assert st.status == sw.SW_OK and st.true_rel_residual <= TOL
    assert oracle_rel_residual(P, phi.cpu().numpy()) <= 1.001 * TOL


def test_ensemble_64_members():
    members = synth.ensemble_members()
    Ps = [synth.problem(nx, ny, seed) for nx, ny, seed in members]
    grids = [grid_for(P) for P in Ps]
    Rs = [torch.as_tensor(P["R"], device="cuda") for P in Ps]
    phis = [torch.zeros_like(R) for R in Rs]
    sts = sw.sw_ensemble_solve(grids, sw.sw_solve_opts_default(prec=sw.SW_PREC_MIXED_FP16, tol=TOL), Rs, phis)
    for P, st, phi in zip(Ps, sts, phis):
        assert st.status == sw.SW_OK
        assert oracle_rel_residual(P, phi.cpu().numpy()) <= 1.001 * TOL


def test_sequence_512x256_warm_start():
    g = None
    phi = torch.zeros((256, 512), dtype=torch.float64, device="cuda")
    o = sw.sw_solve_opts_default(k=4, prec=sw.SW_PREC_MIXED_FP16, tol=TOL, max_iters=2000)
    for t in range(3):
        P = synth.sequence_problem(512, 256, 1000, t)
        if g is None:
            g = grid_for(P)
        else:
            sw.sw_elliptic_set_coeffs(g, *[torch.as_tensor(P[k], device="cuda") for k in sw.COEFF_KEYS])
        st = sw.sw_gcr_solve(g, o, torch.as_tensor(P["R"], device="cuda"), phi)
        assert st.status == sw.SW_OK
        x = phi.cpu().numpy()
        assert oracle_rel_residual(P, x) <= 1.001 * TOL
    ref, _ = O.Problem(P).gcr(P["R"], O.Opts(k=4, tol=1e-13, max_iters=5000))
    assert np.linalg.norm(x - ref) <= 1e-6 * np.linalg.norm(ref)


@pytest.mark.parametrize("row_mode", [1, 2])
@pytest.mark.parametrize("nx,ny,iters", [(1024, 512, 6), (2048, 1024, 5)])
def test_multirow_blocks_fp64_fixed_iterations(nx, ny, iters, row_mode):
    """Grids whose rows outnumber the resident blocks, in both row modes:
    thread blocks that each own several rows (row_mode 1, the instantiation
    built for two resident blocks per SM), and one warp per row (row_mode 2,
    the automatic choice at these widths).  FP64 iterates after a fixed number
    of iterations against the oracle's.

    The bar comes from the conditioning.  One rounding of R (relative 1e-16)
    moves the oracle's own iterates by s: 6e-16 at 512 x 256, 4e-14 at
    1024 x 512, 1e-11 at 2048 x 1024, where the zonal coefficients near the
    poles reach 1e15.  The GPU rounds differently in every operation, so it
    may differ by a hundred such roundings: max(1e-12, 100 s)."""
    P = synth.problem(nx, ny, 5100 + nx)
    g = grid_for(P)
    R = torch.as_tensor(P["R"], device="cuda")
    phi = torch.zeros_like(R)
    o = sw.sw_solve_opts_default(k=4, tol=0.0, max_iters=iters, row_mode=row_mode)
    st = sw.sw_gcr_solve(g, o, R, phi)
    assert st.iterations == iters and st.status == sw.SW_ERR_NOT_CONVERGED
    prob = O.Problem(P)
    oo = O.Opts(k=4, tol=0.0, max_iters=iters, eta=st.eta)
    ref, _ = prob.gcr(P["R"], oo)
    R1 = P["R"] * (1.0 + 1e-16 * np.random.default_rng(1).standard_normal(P["R"].shape))
    ref1, _ = prob.gcr(R1, oo)
    nref = np.linalg.norm(ref)
    s = np.linalg.norm(ref1 - ref) / nref
    err = np.linalg.norm(phi.cpu().numpy() - ref) / nref
    print(f"{nx}x{ny}: GPU vs oracle {err:.2e}, oracle under one rounding of R {s:.2e}")
    assert err <= max(1e-12, 100.0 * s)


def test_largest_grid_4096x2048_mixed():
    """The largest row the library takes (nx = 4096: 256 threads with 16 points
    each in the zonal scans), every block owning many rows.  The oracle
    recomputes the true residual of the GPU's solution."""
    P = synth.problem(4096, 2048, 5300)
    g = grid_for(P)
    R = torch.as_tensor(P["R"], device="cuda")
    phi = torch.zeros_like(R)
    st = sw.sw_gcr_solve(g, sw.sw_solve_opts_default(prec=sw.SW_PREC_MIXED_FP16, tol=TOL, max_iters=6000), R, phi)
    print(f"4096x2048 mixed: {st.iterations} iterations, true residual {st.true_rel_residual:.2e}")
    assert st.status == sw.SW_OK and st.true_rel_residual <= TOL
    assert oracle_rel_residual(P, phi.cpu().numpy()) <= 1.001 * TOL
