"""FP64 CPU oracle of the preconditioned GCR(k) elliptic solve.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library.  It shares no code with
the CUDA path.  See oracle/sw_oracle.c for what each routine computes and the
passage of the paper it follows; the reduced-precision emulation of the
mixed-precision storage plan (Sec. 3.4, Sec. 4.3) is in oracle/emulate.py; the
CNN oracle (learned preconditioner, not in the paper) is in oracle/cnn.py; the
semi-implicit shallow-water time step around the solve (Eqs. 1-10) is in
oracle/swe.py.
"""
from .oracle import *  # noqa: F401,F403
