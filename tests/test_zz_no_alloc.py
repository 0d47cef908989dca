"""sw_gcr_solve_noalloc: the solve with its work vectors in the library's fixed
device scratch.  It gives the results of sw_gcr_solve on the same inputs, call
after call, allocates no device memory, and refuses grids whose workspace does
not fit in the scratch.

This file is collected last, so the scratch is also exercised after every
other GPU test has run in the same process.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16120_gb300 as sw  # noqa: E402

# Both entry points run the same kernel with the same launch shape and fixed
# reduction orders, so the two solutions agree to rounding at most.
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2103_16120_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def grid_with(P, nx, ny):
    g = sw.sw_grid_create(nx, ny)
    sw.sw_elliptic_set_coeffs(g, *[dev(P[k]) for k in sw.COEFF_KEYS])
    return g


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("prec", [sw.SW_PREC_FP64, sw.SW_PREC_MIXED_FP16])
@pytest.mark.parametrize("nx,ny", [(130, 33), (512, 256)])
def test_matches_gcr_solve_on_two_calls_in_a_row(nx, ny, prec):
    P = synth.problem(nx, ny, 4100 + nx)
    R2 = synth.problem(nx, ny, 4200 + nx)["R"]
    g_ref, g = grid_with(P, nx, ny), grid_with(P, nx, ny)
    o = sw.sw_solve_opts_default(prec=prec, tol=1e-8)
    for R in (P["R"], R2):
        Rd = dev(R)
        ref = torch.zeros_like(Rd)
        st_ref = sw.sw_gcr_solve(g_ref, o, Rd, ref)
        phi = torch.zeros_like(Rd)
        st = sw.sw_gcr_solve_noalloc(g, o, Rd, phi)
        torch.cuda.synchronize()
        assert st.status == st_ref.status == sw.SW_OK
        assert st.iterations == st_ref.iterations
        assert rel(phi, ref) <= TOL
        assert abs(st.true_rel_residual - st_ref.true_rel_residual) <= 1e-14


def test_matches_gcr_solve_when_blocks_own_several_rows():
    """512 rows of 512 points with 256 threads per row are more rows than the
    device holds resident blocks, so every block cycles over several rows and
    the launch may take the two-blocks-per-SM kernel.  The scratch call must
    take the same launch shape as sw_gcr_solve."""
    nx, ny = 512, 512
    P = synth.problem(nx, ny, 4500)
    g_ref, g = grid_with(P, nx, ny), grid_with(P, nx, ny)
    o = sw.sw_solve_opts_default(prec=sw.SW_PREC_MIXED_FP16, tol=1e-8, k=2, threads_per_row=256)
    assert sw.sw_grid_workspace_bytes(g, o) <= sw.SW_NOALLOC_SCRATCH_BYTES
    props = torch.cuda.get_device_properties(0)
    assert ny > 2 * props.multi_processor_count
    Rd = dev(P["R"])
    for _ in range(2):
        ref = torch.zeros_like(Rd)
        st_ref = sw.sw_gcr_solve(g_ref, o, Rd, ref)
        phi = torch.zeros_like(Rd)
        st = sw.sw_gcr_solve_noalloc(g, o, Rd, phi)
        torch.cuda.synchronize()
        assert st.status == st_ref.status == sw.SW_OK
        assert st.iterations == st_ref.iterations
        assert rel(phi, ref) <= TOL


def test_allocates_no_device_memory():
    nx, ny = 512, 256
    P = synth.problem(nx, ny, 4300)
    Rd = dev(P["R"])
    phis = [torch.zeros_like(Rd) for _ in range(4)]
    g_setup, g, g_alloc = grid_with(P, nx, ny), grid_with(P, nx, ny), grid_with(P, nx, ny)
    o = sw.sw_solve_opts_default(prec=sw.SW_PREC_FP64, tol=1e-8)
    sw.sw_gcr_solve_noalloc(g_setup, o, Rd, phis[0])     # first call on the device: one-time set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    sw.sw_gcr_solve_noalloc(g, o, Rd, phis[1])
    sw.sw_gcr_solve_noalloc(g, o, Rd, phis[2])
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    # the same measurement does see the workspace that sw_gcr_solve allocates
    # for a grid on its first solve
    sw.sw_gcr_solve(g_alloc, o, Rd, phis[3])
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] >= sw.sw_grid_workspace_bytes(g_alloc, o)


def test_rejects_workspace_beyond_the_scratch():
    nx, ny = 512, 256
    P = synth.problem(nx, ny, 4400)
    g = grid_with(P, nx, ny)
    Rd = dev(P["R"])
    fits = sw.sw_solve_opts_default(prec=sw.SW_PREC_FP64, k=4)
    too_big = sw.sw_solve_opts_default(prec=sw.SW_PREC_FP64, k=8)
    assert sw.sw_grid_workspace_bytes(g, fits) <= sw.SW_NOALLOC_SCRATCH_BYTES
    assert sw.sw_grid_workspace_bytes(g, too_big) > sw.SW_NOALLOC_SCRATCH_BYTES
    phi = torch.zeros_like(Rd)
    with pytest.raises(sw.SwError) as ei:
        sw.sw_gcr_solve_noalloc(g, too_big, Rd, phi)
    assert ei.value.status == sw.SW_ERR_INVALID_ARG
    assert "bytes of scratch" in str(ei.value)
    assert float(phi.abs().max()) == 0.0          # rejected before anything ran
