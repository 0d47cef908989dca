"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 path: every kernel and the full GCR at fixed iteration counts and when
converged agree with the oracle to 1e-12 relative L2 (rounding order is the
only difference).  Mixed precision: the same true FP64 residual is reached
and the solution error against the oracle is at most 1e-6 relative L2.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16120_gb300 as sw  # noqa: E402

FP64_TOL = 1e-12


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def make(nx, ny, seed, **kw):
    P = synth.problem(nx, ny, seed, **kw)
    g = sw.sw_grid_create(nx, ny)
    co = [dev(P[k]) for k in sw.COEFF_KEYS]
    sw.sw_elliptic_set_coeffs(g, *co)
    return P, g, co


def oracle_opts(o: "sw.SolveOpts", eta):
    return O.Opts(k=o.k, tol=o.tol, max_iters=o.max_iters, min_iters=o.min_iters, pc=o.pc,
                  n_rich=o.n_richardson, eta=eta, omega=o.omega, ru_every=o.ru_every)


SIZES = [(4, 2), (16, 8), (34, 9), (128, 64), (130, 33), (512, 256)]


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2103_16120_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("nx,ny", SIZES)
def test_operator_fp64_and_fp32(nx, ny):
    P, g, co = make(nx, ny, 100 + nx)
    rng = np.random.default_rng(nx * 7 + ny)
    x = rng.standard_normal((ny, nx)) * 10
    ref = O.Problem(P).operator(x)
    y = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    sw.sw_operator_apply(g, dev(x), y)
    assert rel(y.cpu().numpy(), ref) <= FP64_TOL
    y32 = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
    sw.sw_operator_apply(g, dev(x, torch.float32), y32)
    # FP32 coefficients and arithmetic: a few units of 2^-24 per term, with the
    # usual cancellation of the stencil
    assert rel(y32.cpu().numpy(), ref) <= 1e-5


def test_operator_full_size_sampled():
    """2048 x 1024 (the large single-grid size) in the library's launch
    configuration: the oracle computes the full result on the host."""
    P, g, co = make(2048, 1024, 4000)
    x = np.random.default_rng(1).standard_normal((1024, 2048))
    ref = O.Problem(P).operator(x)
    y = torch.empty_like(dev(x))
    sw.sw_operator_apply(g, dev(x), y)
    assert rel(y.cpu().numpy(), ref) <= FP64_TOL


@pytest.mark.parametrize("nx,ny", [(16, 8), (130, 33), (512, 256)])
def test_eta_matches_oracle(nx, ny):
    P, g, co = make(nx, ny, 200 + nx)
    assert abs(sw.sw_grid_get_eta(g) / O.Problem(P).eta_auto() - 1) <= FP64_TOL


@pytest.mark.parametrize("pc,nrich", [(0, 1), (1, 1), (2, 1), (2, 3), (3, 1), (3, 2), (3, 5)])
@pytest.mark.parametrize("nx,ny", [(4, 2), (34, 9), (128, 64), (512, 256)])
def test_precond_fp64(pc, nrich, nx, ny):
    P, g, co = make(nx, ny, 300 + nx + pc)
    r = np.random.default_rng(pc * 31 + nrich).standard_normal((ny, nx)) * 1e3
    o = sw.sw_solve_opts_default(pc=pc, n_richardson=nrich, omega=0.7)
    q = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    sw.sw_precond_apply(g, o, dev(r), q)
    eta = sw.sw_grid_get_eta(g)
    ref = O.Problem(P).precond(r, oracle_opts(o, eta), eta=eta)
    assert rel(q.cpu().numpy(), ref) <= FP64_TOL


@pytest.mark.parametrize("prec", [sw.SW_PREC_MIXED_FP16, sw.SW_PREC_MIXED_BF16])
@pytest.mark.parametrize("nx,ny", [(34, 9), (256, 128)])
def test_precond_mixed(prec, nx, ny):
    P, g, co = make(nx, ny, 400 + nx)
    r = np.random.default_rng(5).standard_normal((ny, nx)) * 1e3
    o = sw.sw_solve_opts_default(prec=prec)
    q = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
    sw.sw_precond_apply(g, o, dev(r, torch.float32), q)
    eta = sw.sw_grid_get_eta(g)
    ref = O.Problem(P).precond(r, oracle_opts(o, eta), eta=eta)
    # 16-bit storage of q between the sweeps and of the output: 2^-11 (FP16)
    # or 2^-8 (BF16) relative to the row maximum, per stored value
    tol = 4e-3 if prec == sw.SW_PREC_MIXED_FP16 else 3e-2
    assert rel(q.cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("iters", [1, 2, 4, 5, 12])
@pytest.mark.parametrize("nx,ny,k", [(16, 8, 4), (130, 33, 3), (256, 128, 4)])
def test_gcr_fp64_fixed_iterations(iters, nx, ny, k):
    P, g, co = make(nx, ny, 500 + nx)
    R = dev(P["R"])
    phi = torch.zeros_like(R)
    o = sw.sw_solve_opts_default(k=k, tol=0.0, max_iters=iters)
    st = sw.sw_gcr_solve(g, o, R, phi)
    assert st.iterations == iters and st.status == sw.SW_ERR_NOT_CONVERGED
    ref, rs = O.Problem(P).gcr(P["R"], oracle_opts(o, st.eta))
    assert rel(phi.cpu().numpy(), ref) <= FP64_TOL
    # residual norms relative to ||R||: rounding of r = L(phi) - R is ~1e-16 ||R||
    assert abs(st.true_rel_residual - rs["true_rel_residual"]) <= 1e-10 * rs["true_rel_residual"] + 1e-14


@pytest.mark.parametrize("pc", [0, 1, 2, 3])
def test_gcr_fp64_converged_all_options(pc):
    P, g, co = make(64, 32, 600 + pc)
    R = dev(P["R"])
    phi = torch.zeros_like(R)
    o = sw.sw_solve_opts_default(pc=pc, tol=1e-10, max_iters=2000, n_richardson=2)
    st = sw.sw_gcr_solve(g, o, R, phi)
    ref, rs = O.Problem(P).gcr(P["R"], oracle_opts(o, st.eta))
    assert st.status == sw.SW_OK and st.converged == 1
    assert st.iterations == rs["iterations"]
    assert rel(phi.cpu().numpy(), ref) <= FP64_TOL
    assert st.true_rel_residual <= 1e-10


def test_gcr_fp64_warm_start_ru_every_min_iters_history():
    P, g, co = make(128, 64, 700)
    R = dev(P["R"])
    phi0 = np.random.default_rng(2).standard_normal((64, 128))
    phi = dev(phi0)
    hist = torch.empty(61, dtype=torch.float64, device="cuda")
    rowres = torch.empty(64, dtype=torch.float64, device="cuda")
    o = sw.sw_solve_opts_default(tol=1e-9, max_iters=60, min_iters=6, ru_every=3,
                                 res_history=hist, row_residual=rowres)
    st = sw.sw_gcr_solve(g, o, R, phi)
    ref, rs, h_ref, _ = O.Problem(P).gcr(P["R"], oracle_opts(o, st.eta), phi0=phi0, want_history=True)
    assert st.iterations == rs["iterations"] and st.status == sw.SW_OK
    assert rel(phi.cpu().numpy(), ref) <= FP64_TOL
    h = hist.cpu().numpy()[: st.iterations + 1]
    # history entries are ||r|| / ||R||; rounding in r is ~1e-16 ||R|| absolute
    assert np.allclose(h, h_ref, rtol=1e-9, atol=1e-13)
    assert np.all(np.isnan(hist.cpu().numpy()[st.iterations + 1:]))
    r = O.Problem(P).operator(phi.cpu().numpy()) - P["R"]
    nR = np.linalg.norm(P["R"])
    assert np.allclose(rowres.cpu().numpy(), np.sqrt(np.sum(r * r, axis=1)), rtol=1e-9, atol=1e-13 * nR)


def test_gcr_zero_rhs_and_exact_guess():
    P, g, co = make(32, 16, 800)
    phi = dev(np.ones((16, 32)))
    st = sw.sw_gcr_solve(g, sw.sw_solve_opts_default(), torch.zeros_like(phi), phi)
    assert st.status == sw.SW_OK and st.iterations == 0 and float(phi.abs().max()) == 0.0
    ex, _ = O.Problem(P).gcr(P["R"], O.Opts(tol=1e-13))
    phi = dev(ex)
    st = sw.sw_gcr_solve(g, sw.sw_solve_opts_default(tol=1e-8), dev(P["R"]), phi)
    assert st.iterations == 0 and st.status == sw.SW_OK


@pytest.mark.parametrize("prec", [sw.SW_PREC_MIXED_FP16, sw.SW_PREC_MIXED_BF16])
@pytest.mark.parametrize("nx,ny", [(128, 64), (512, 256)])
def test_gcr_mixed_reaches_tolerance(prec, nx, ny):
    P, g, co = make(nx, ny, 900 + nx)
    R = dev(P["R"])
    phi = torch.zeros_like(R)
    o = sw.sw_solve_opts_default(prec=prec, tol=1e-8, max_iters=400, ru_every=0)
    st = sw.sw_gcr_solve(g, o, R, phi)
    assert st.status == sw.SW_OK, st.as_dict()
    assert st.true_rel_residual <= 1e-8
    # independent check of the true residual with the oracle operator
    prob = O.Problem(P)
    x = phi.cpu().numpy()
    assert np.linalg.norm(prob.operator(x) - P["R"]) <= 1e-8 * np.linalg.norm(P["R"]) * (1 + 1e-9)
    ref, rs = prob.gcr(P["R"], O.Opts(tol=1e-12, max_iters=2000))
    assert rel(x, ref) <= 1e-6


def test_ensemble_matches_single_solves():
    members = [(64, 32, 11), (128, 64, 12), (34, 9, 13), (64, 32, 14)]
    grids, Rs, phis, keep = [], [], [], []
    for nx, ny, seed in members:
        P, g, co = make(nx, ny, seed)
        grids.append(g); Rs.append(dev(P["R"])); phis.append(torch.zeros_like(Rs[-1])); keep.append((P, co))
    o = sw.sw_solve_opts_default(tol=1e-10, max_iters=500)
    stats = sw.sw_ensemble_solve(grids, o, Rs, phis)
    for (P, _), g, phi, st in zip(keep, grids, phis, stats):
        assert st.status == sw.SW_OK
        ref, rs = O.Problem(P).gcr(P["R"], oracle_opts(o, st.eta))
        assert st.iterations == rs["iterations"]
        assert rel(phi.cpu().numpy(), ref) <= FP64_TOL


def test_invalid_arguments_raise():
    P, g, co = make(16, 8, 1)
    R = dev(P["R"])
    phi = torch.zeros_like(R)
    with pytest.raises(sw.SwError):
        sw.sw_gcr_solve(g, sw.sw_solve_opts_default(k=0), R, phi)
    with pytest.raises(sw.SwError):
        sw.sw_gcr_solve(g, sw.sw_solve_opts_default(prec=7), R, phi)
    with pytest.raises(sw.SwError):
        sw.sw_operator_apply(g, R, R)          # in-place (overlapping) call
    g2 = sw.sw_grid_create(16, 8)
    with pytest.raises(sw.SwError):            # no coefficients yet
        sw.sw_gcr_solve(g2, sw.sw_solve_opts_default(), R, phi)
    with pytest.raises(sw.SwError):            # the same grid twice
        sw.sw_ensemble_solve([g, g], sw.sw_solve_opts_default(), [R, R], [phi, torch.zeros_like(R)])


def test_nonfinite_input_reported():
    P, g, co = make(16, 8, 2)
    R = P["R"].copy()
    R[3, 5] = np.nan
    phi = torch.zeros((8, 16), dtype=torch.float64, device="cuda")
    st = sw.sw_gcr_solve(g, sw.sw_solve_opts_default(), dev(R), phi)
    assert st.status == sw.SW_ERR_NONFINITE
