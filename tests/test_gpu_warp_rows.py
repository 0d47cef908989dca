"""The solver kernel with one warp per latitude row (row_mode 2, the automatic
choice for large grids of a power-of-two width) against the FP64 CPU oracle and
against the thread-block row mode.

FP64: iterates at fixed iteration counts and converged solutions within
1e-12 of the oracle, for every preconditioner option, the pole rows and a
row count that is not a multiple of the warps.  Mixed precision: the FP64
true residual reaches the tolerance, the solution is within 1e-6 of the
oracle's, and the iteration count is that of the block mode within a few
(the inner products sum in another order); the row lengths give zonal-solve
chunks of 4 to 64 points per lane.
"""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16120_gb300 as sw  # noqa: E402

FP64_TOL = 1e-12
WARP, BLOCK = 2, 1


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2103_16120_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def make(nx, ny, seed):
    P = synth.problem(nx, ny, seed)
    g = sw.sw_grid_create(nx, ny)
    sw.sw_elliptic_set_coeffs(g, *[dev(P[k]) for k in sw.COEFF_KEYS])
    return P, g


def oracle_opts(o, eta):
    return O.Opts(k=o.k, tol=o.tol, max_iters=o.max_iters, min_iters=o.min_iters, pc=o.pc,
                  n_rich=o.n_richardson, eta=eta, omega=o.omega, ru_every=o.ru_every)


@pytest.mark.parametrize("iters", [1, 4, 12])
@pytest.mark.parametrize("nx,ny,k", [(128, 64, 4), (256, 37, 3), (512, 96, 4)])
def test_fp64_fixed_iterations(iters, nx, ny, k):
    P, g = make(nx, ny, 6100 + nx + ny)
    R = dev(P["R"])
    phi = torch.zeros_like(R)
    o = sw.sw_solve_opts_default(k=k, tol=0.0, max_iters=iters, row_mode=WARP)
    st = sw.sw_gcr_solve(g, o, R, phi)
    assert st.iterations == iters and st.status == sw.SW_ERR_NOT_CONVERGED
    ref, rs = O.Problem(P).gcr(P["R"], oracle_opts(o, st.eta))
    assert rel(phi.cpu().numpy(), ref) <= FP64_TOL
    assert abs(st.true_rel_residual - rs["true_rel_residual"]) <= 1e-10 * rs["true_rel_residual"] + 1e-14


@pytest.mark.parametrize("pc,nrich", [(0, 1), (1, 1), (2, 2), (3, 1), (3, 2), (3, 3)])
def test_fp64_converged_every_option(pc, nrich):
    P, g = make(128, 48, 6200 + pc)
    R = dev(P["R"])
    phi = torch.zeros_like(R)
    o = sw.sw_solve_opts_default(pc=pc, n_richardson=nrich, tol=1e-10, max_iters=3000, row_mode=WARP)
    st = sw.sw_gcr_solve(g, o, R, phi)
    ref, rs = O.Problem(P).gcr(P["R"], oracle_opts(o, st.eta))
    assert st.status == sw.SW_OK and st.iterations == rs["iterations"]
    assert rel(phi.cpu().numpy(), ref) <= FP64_TOL


def test_fp64_warm_start_history_row_residual():
    P, g = make(256, 64, 6300)
    R = dev(P["R"])
    phi0 = np.random.default_rng(3).standard_normal((64, 256))
    phi = dev(phi0)
    hist = torch.empty(81, dtype=torch.float64, device="cuda")
    rowres = torch.empty(64, dtype=torch.float64, device="cuda")
    o = sw.sw_solve_opts_default(tol=1e-9, max_iters=80, min_iters=5, ru_every=3, res_history=hist,
                                 row_residual=rowres, row_mode=WARP)
    st = sw.sw_gcr_solve(g, o, R, phi)
    ref, rs, h_ref, _ = O.Problem(P).gcr(P["R"], oracle_opts(o, st.eta), phi0=phi0, want_history=True)
    assert st.status == sw.SW_OK and st.iterations == rs["iterations"]
    assert rel(phi.cpu().numpy(), ref) <= FP64_TOL
    assert np.allclose(hist.cpu().numpy()[: st.iterations + 1], h_ref, rtol=1e-9, atol=1e-13)
    r = O.Problem(P).operator(phi.cpu().numpy()) - P["R"]
    assert np.allclose(rowres.cpu().numpy(), np.sqrt(np.sum(r * r, axis=1)), rtol=1e-9,
                       atol=1e-13 * np.linalg.norm(P["R"]))


@pytest.mark.parametrize("prec", [sw.SW_PREC_MIXED_FP16, sw.SW_PREC_MIXED_BF16])
@pytest.mark.parametrize("nx,ny", [(128, 64), (512, 256), (1024, 48), (2048, 40)])
def test_mixed_matches_block_mode_and_oracle(prec, nx, ny):
    P, g = make(nx, ny, 6400 + nx)
    R = dev(P["R"])
    out = {}
    for mode in (BLOCK, WARP):
        phi = torch.zeros_like(R)
        o = sw.sw_solve_opts_default(prec=prec, tol=1e-8, max_iters=2000, row_mode=mode)
        st = sw.sw_gcr_solve(g, o, R, phi)
        assert st.status == sw.SW_OK and st.true_rel_residual <= 1e-8, st.as_dict()
        out[mode] = (st, phi.cpu().numpy())
    prob = O.Problem(P)
    x = out[WARP][1]
    assert np.linalg.norm(prob.operator(x) - P["R"]) <= 1e-8 * np.linalg.norm(P["R"]) * (1 + 1e-9)
    ref, _ = prob.gcr(P["R"], O.Opts(tol=1e-12, max_iters=4000))
    assert rel(x, ref) <= 1e-6
    assert abs(out[WARP][0].iterations - out[BLOCK][0].iterations) <= 3


def test_row_mode_checks():
    P, g = make(130, 33, 6500)
    R = dev(P["R"])
    with pytest.raises(sw.SwError) as ei:
        sw.sw_gcr_solve(g, sw.sw_solve_opts_default(row_mode=WARP), R, torch.zeros_like(R))
    assert ei.value.status == sw.SW_ERR_INVALID_ARG
    P2, g2 = make(128, 16, 6501)
    with pytest.raises(sw.SwError):
        sw.sw_gcr_solve(g2, sw.sw_solve_opts_default(row_mode=3), dev(P2["R"]), torch.zeros_like(dev(P2["R"])))
    # block mode on the same grid still works
    st = sw.sw_gcr_solve(g, sw.sw_solve_opts_default(row_mode=BLOCK, tol=1e-8), R, torch.zeros_like(R))
    assert st.status == sw.SW_OK
