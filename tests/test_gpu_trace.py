"""The device time line (paper_2103_16120_gb300.trace) of the traced build:
the same solve as the release build (same iterations), with the phase tags of
every iteration recorded."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16120_gb300 as sw  # noqa: E402
import synth  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_timeline_of_the_traced_build():
    from paper_2103_16120_gb300 import build
    build.build()
    nx, ny = 128, 64
    r = subprocess.run([sys.executable, "-m", "paper_2103_16120_gb300.trace", str(nx), str(ny), "1", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    t = json.loads(r.stdout.strip().splitlines()[-1])
    P = synth.problem(nx, ny, 1000)
    g = sw.sw_grid_create(nx, ny)
    sw.sw_elliptic_set_coeffs(g, *[torch.as_tensor(P[k], device="cuda") for k in sw.COEFF_KEYS])
    R = torch.as_tensor(P["R"], device="cuda")
    st = sw.sw_gcr_solve(g, sw.sw_solve_opts_default(prec=1, tol=1e-8, max_iters=5000), R, torch.zeros_like(R))
    assert t["iterations"] == st.iterations
    # every update, Richardson stage and L(e) phase of every iteration
    n = t["ns"]
    assert n["11->201"][0] == n["12->301"][0] == n["13->101"][0] == st.iterations
