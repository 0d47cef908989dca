"""Ensembles in one persistent launch: the asynchronous entry point, its
capture in a CUDA graph, and the launch-shape autotuner, each against the
synchronous sw_ensemble_solve on the same members (same kernel, same launch
shape, fixed reduction orders: equal results)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16120_gb300 as sw  # noqa: E402
from paper_2103_16120_gb300 import autotune  # noqa: E402

MEMBERS = [(128, 64, 9001), (128, 64, 9002), (256, 128, 9003), (130, 33, 9004), (512, 256, 9005)]


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2103_16120_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def members():
    Ps = [synth.problem(nx, ny, seed) for nx, ny, seed in MEMBERS]
    grids = []
    for (nx, ny, _), P in zip(MEMBERS, Ps):
        g = sw.sw_grid_create(nx, ny)
        sw.sw_elliptic_set_coeffs(g, *[torch.as_tensor(P[k], device="cuda") for k in sw.COEFF_KEYS])
        grids.append(g)
    Rs = [torch.as_tensor(P["R"], device="cuda") for P in Ps]
    return grids, Rs


@pytest.mark.parametrize("prec", [sw.SW_PREC_FP64, sw.SW_PREC_MIXED_FP16])
def test_async_equals_sync(prec):
    grids, Rs = members()
    o = sw.sw_solve_opts_default(prec=prec, tol=1e-8)
    ref = [torch.zeros_like(R) for R in Rs]
    sts = sw.sw_ensemble_solve(grids, o, Rs, ref)
    phis = [torch.zeros_like(R) for R in Rs]
    buf = sw.stats_buffer(len(grids))
    sw.sw_ensemble_solve_async(grids, o, Rs, phis, buf)
    torch.cuda.synchronize()
    got = sw.stats_from_device(buf, len(grids))
    for a, b, p, q in zip(sts, got, ref, phis):
        assert a.status == b.status == sw.SW_OK
        assert a.iterations == b.iterations
        assert a.true_rel_residual == b.true_rel_residual and a.eta == b.eta
        assert torch.equal(p, q)


def test_back_to_back_async_solves_of_one_grid():
    """A warm-started sequence enqueued without synchronisation: with one
    member each call's descriptors are kernel parameters of its launch, so
    later calls cannot overwrite what an earlier, not yet executed, launch
    reads.  Each step between the solves changes the coefficients too."""
    nx, ny, n = 256, 128, 7
    Ps = [synth.sequence_problem(nx, ny, 9100, t) for t in range(n)]
    cos = [[torch.as_tensor(P[k], device="cuda") for k in sw.COEFF_KEYS] for P in Ps]
    Rs = [torch.as_tensor(P["R"], device="cuda") for P in Ps]
    o = sw.sw_solve_opts_default(prec=sw.SW_PREC_MIXED_FP16, tol=1e-8)
    g = sw.sw_grid_create(nx, ny)
    ref, phi = [], torch.zeros_like(Rs[0])
    for t in range(n):
        sw.sw_elliptic_set_coeffs(g, *cos[t])
        st = sw.sw_gcr_solve(g, o, Rs[t], phi)
        assert st.status == sw.SW_OK
        ref.append((phi.clone(), st.iterations))
    bufs = [sw.stats_buffer(1) for _ in range(n)]
    outs, phi = [], torch.zeros_like(Rs[0])
    torch.cuda.synchronize()
    for t in range(n):
        sw.sw_elliptic_set_coeffs(g, *cos[t])
        sw.sw_ensemble_solve_async([g], o, [Rs[t]], [phi], bufs[t])
        outs.append(phi.clone())                          # stream-ordered copy
    torch.cuda.synchronize()
    for t in range(n):
        got = sw.stats_from_device(bufs[t], 1)[0]
        assert got.status == sw.SW_OK and got.iterations == ref[t][1]
        assert torch.equal(outs[t], ref[t][0])


def test_graph_capture_and_replay():
    grids, Rs = members()
    o = sw.sw_solve_opts_default(prec=sw.SW_PREC_MIXED_FP16, tol=1e-8)
    ref = [torch.zeros_like(R) for R in Rs]
    sts = sw.sw_ensemble_solve(grids, o, Rs, ref)            # also sizes the workspaces
    phis = [torch.zeros_like(R) for R in Rs]
    buf = sw.stats_buffer(len(grids))
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            for p in phis:
                p.zero_()
            sw.sw_ensemble_solve_async(grids, o, Rs, phis, buf)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        for p in phis:
            p.fill_(1.0)                                       # replays start from zero again
        graph.replay()
        torch.cuda.synchronize()
        got = sw.stats_from_device(buf, len(grids))
        for a, b, p, q in zip(sts, got, ref, phis):
            assert b.status == sw.SW_OK and a.iterations == b.iterations
            assert torch.equal(p, q)


def test_autotuner_picks_a_width_and_caches_it():
    grids, Rs = members()
    o = sw.sw_solve_opts_default(prec=sw.SW_PREC_MIXED_FP16, tol=1e-8)
    phis = [torch.zeros_like(R) for R in Rs]
    best, table = autotune.tune_ensemble(grids, o, Rs, phis)
    assert best.threads_per_row in table and np.isfinite(table[best.threads_per_row])
    assert all(float(p.abs().max()) == 0.0 for p in phis)     # first guesses restored
    again, table2 = autotune.tune_ensemble(grids, o, Rs, phis)
    assert again.threads_per_row == best.threads_per_row and table2 is table
    sts = sw.sw_ensemble_solve(grids, best, Rs, phis)
    assert all(s.status == sw.SW_OK and s.true_rel_residual <= 1e-8 for s in sts)


def test_one_member_graph_replays_with_new_right_hand_sides():
    """One member: the descriptors are kernel parameters recorded in the graph.
    Replays after new contents of R (the same buffer) give the direct solves'
    results, and a direct call on the same grid between replays, into another
    buffer, disturbs neither."""
    nx, ny = 256, 128
    Ps = [synth.sequence_problem(nx, ny, 9200, t) for t in range(3)]
    g = sw.sw_grid_create(nx, ny)
    sw.sw_elliptic_set_coeffs(g, *[torch.as_tensor(Ps[0][k], device="cuda") for k in sw.COEFF_KEYS])
    o = sw.sw_solve_opts_default(prec=sw.SW_PREC_MIXED_FP16, tol=1e-8)
    Rs = [torch.as_tensor(P["R"], device="cuda") for P in Ps]
    ref = []
    for Rt in Rs:
        x = torch.zeros_like(Rt)
        st = sw.sw_gcr_solve(g, o, Rt, x)
        assert st.status == sw.SW_OK
        ref.append((x, st.iterations))
    R = Rs[0].clone()
    phi = torch.zeros_like(R)
    buf = sw.stats_buffer(1)
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            phi.zero_()
            sw.sw_ensemble_solve_async([g], o, [R], [phi], buf)
    torch.cuda.current_stream().wait_stream(s)
    for t in (2, 0, 1):
        R.copy_(Rs[t])
        graph.replay()
        other, obuf = torch.zeros_like(R), sw.stats_buffer(1)
        sw.sw_ensemble_solve_async([g], o, [Rs[t]], [other], obuf)
        torch.cuda.synchronize()
        got = sw.stats_from_device(buf, 1)[0]
        assert got.status == sw.SW_OK and got.iterations == ref[t][1]
        assert torch.equal(phi, ref[t][0]) and torch.equal(other, ref[t][0])
        assert sw.stats_from_device(obuf, 1)[0].iterations == ref[t][1]


@pytest.mark.parametrize("prec", [sw.SW_PREC_MIXED_FP16, sw.SW_PREC_FP64])
def test_warp_rows_ensemble_matches_the_oracle_and_block_mode(prec):
    """An ensemble whose grids all have power-of-two widths runs with one warp
    per row (row_mode 2; the automatic choice for the mixed precisions),
    members sharing the resident blocks by work.  Each member reaches the FP64
    true residual and the oracle's solution, and the thread-block mode (the
    same method, other reduction groupings) agrees to the tolerance."""
    import oracle as O
    spec = [(128, 64, 9101), (128, 64, 9102), (256, 128, 9103), (512, 256, 9104), (256, 96, 9105)]
    Ps = [synth.problem(nx, ny, seed) for nx, ny, seed in spec]
    grids = []
    for (nx, ny, _), P in zip(spec, Ps):
        g = sw.sw_grid_create(nx, ny)
        sw.sw_elliptic_set_coeffs(g, *[torch.as_tensor(P[k], device="cuda") for k in sw.COEFF_KEYS])
        grids.append(g)
    Rs = [torch.as_tensor(P["R"], device="cuda") for P in Ps]
    out = {}
    for mode in (1, 2):
        o = sw.sw_solve_opts_default(prec=prec, tol=1e-8, max_iters=3000, row_mode=mode)
        phis = [torch.zeros_like(R) for R in Rs]
        sts = sw.sw_ensemble_solve(grids, o, Rs, phis)
        for st in sts:
            assert st.status == sw.SW_OK and st.true_rel_residual <= 1e-8, st.as_dict()
        out[mode] = [p.cpu().numpy() for p in phis]
    for P, x2, x1 in zip(Ps, out[2], out[1]):
        ref, _ = O.Problem(P).gcr(P["R"], O.Opts(tol=1e-12, max_iters=4000))
        # both stop at a residual of 1e-8; the conditioning turns that into a
        # solution error of up to a few 1e-7
        tol = 1e-6
        assert np.linalg.norm(x2 - ref) <= tol * np.linalg.norm(ref)
        assert np.linalg.norm(x2 - x1) <= 2 * tol * np.linalg.norm(ref)
