"""Failure detection without a GPU fault: a solver barrier that waits for an
arrival nothing provides runs out after its (shortened) limit.  The solve
returns SW_ERR_TIMEOUT, the CUDA context stays usable, and the next solve
succeeds."""
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16120_gb300 as sw  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2103_16120_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def test_barrier_timeout_is_reported_and_recoverable():
    nx, ny = 128, 64
    P = synth.problem(nx, ny, 9100)
    g = sw.sw_grid_create(nx, ny)
    sw.sw_elliptic_set_coeffs(g, *[torch.as_tensor(P[k], device="cuda") for k in sw.COEFF_KEYS])
    R = torch.as_tensor(P["R"], device="cuda")
    o = sw.sw_solve_opts_default(prec=sw.SW_PREC_MIXED_FP16, tol=1e-8)
    try:
        sw.sw_debug_barrier(1, 0.05)           # one arrival that never comes; 50 ms limit
        phi = torch.zeros_like(R)
        with pytest.raises(sw.SwError) as ei:
            sw.sw_gcr_solve(g, o, R, phi)
        assert ei.value.status == sw.SW_ERR_TIMEOUT
        assert "barrier" in str(ei.value)
    finally:
        sw.sw_debug_barrier(0, 0.0)
    # the context is intact: the same solve now converges
    phi = torch.zeros_like(R)
    st = sw.sw_gcr_solve(g, o, R, phi)
    assert st.status == sw.SW_OK and st.true_rel_residual <= 1e-8
    torch.cuda.synchronize()
