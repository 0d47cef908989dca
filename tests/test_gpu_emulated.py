"""The mixed-precision GPU solve against the reduced-precision emulation
(oracle/emulate.py) of its own storage plan.

A mixed result has no bit pattern to match: the FP32 arithmetic and the order
of the sums differ from the emulation's (parity unpinned).  What the emulation
fixes is the behaviour of the storage plan, so the checks are statistical,
over seeded problems of the benchmark's grids:
* the GPU's iteration count is within one of the emulation's on at least 90 %
  of the seeds, and never more than three away;
* the GPU's solution error against the FP64 oracle is within a factor of ten
  of the emulation's (both are set by the tolerance, not by the format).
"""
import numpy as np
import pytest

import oracle as O
from oracle import emulate as E
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16120_gb300 as sw  # noqa: E402

TOL = 1e-8
CASES = [(128, 64, 9000 + s) for s in range(16)] + [(256, 128, 9100 + s) for s in range(8)] + \
        [(512, 256, 9200 + s) for s in range(4)]


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2103_16120_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def gpu_solve(P, prec):
    ny, nx = P["C"].shape
    g = sw.sw_grid_create(nx, ny)
    sw.sw_elliptic_set_coeffs(g, *[torch.as_tensor(P[k], device="cuda") for k in sw.COEFF_KEYS])
    R = torch.as_tensor(P["R"], device="cuda")
    phi = torch.zeros_like(R)
    st = sw.sw_gcr_solve(g, sw.sw_solve_opts_default(k=4, prec=prec, tol=TOL, max_iters=400), R, phi)
    assert st.status == sw.SW_OK
    return st.iterations, phi.cpu().numpy()


@pytest.mark.parametrize("prec,qfmt", [(sw.SW_PREC_MIXED_FP16, "fp16"), (sw.SW_PREC_MIXED_BF16, "bf16")])
def test_iterations_and_error_follow_the_emulation(prec, qfmt):
    close, rows = 0, []
    for nx, ny, seed in CASES:
        P = synth.problem(nx, ny, seed)
        exact, _ = O.Problem(P).gcr(P["R"], O.Opts(k=4, tol=1e-13, max_iters=5000))
        phe, se = E.MixedSolve(P, qfmt=qfmt).solve(P["R"], O.Opts(k=4, tol=TOL, max_iters=400))
        assert se["converged"] == 1
        itg, phg = gpu_solve(P, prec)
        nrm = np.linalg.norm(exact)
        eg, ee = np.linalg.norm(phg - exact) / nrm, np.linalg.norm(phe - exact) / nrm
        rows.append((nx, ny, seed, itg, se["iterations"], eg, ee))
        close += abs(itg - se["iterations"]) <= 1
        assert abs(itg - se["iterations"]) <= 3, rows[-1]
        assert 0.1 * ee <= eg <= 10 * ee, rows[-1]
    for r in rows:
        print("%4dx%-4d seed %d: GPU %3d its, emulated %3d; error %.2e / %.2e" % r)
    assert close >= 0.9 * len(CASES)
