"""Seeded synthetic inputs for the elliptic solve on the longitude/latitude sphere.

This package builds the *inputs* of the Helmholtz problem L(Phi) = R (Eqs. 9-10):
the seven coefficient fields A11, A12, A21, A22, B1, B2, C and the right-hand
side R, from a seeded synthetic shallow-water state.  It contains no solver
arithmetic (no operator application, no preconditioner, no Krylov step) and is
the only code shared by the CUDA path's tests/benchmarks and the CPU oracle.

Layout of every field: numpy float64 array of shape (ny, nx), row j is the
latitude phi_j = -pi/2 + (j + 1/2) * pi/ny, column i the longitude
lambda_i = 2*pi*i/nx (longitude contiguous).
"""
from .sphere import grid_coords, real_sh, random_sh_field  # noqa: F401
from .shallow_water import (  # noqa: F401
    EARTH, SWState, synthetic_state, coefficients, rhs_divergence, problem,
    sequence_problem, ensemble_members, random_rhs,
)
from .model_state import (  # noqa: F401
    ModelState, balanced_zonal_state, gravity_mode_state, perturbed_state, paper_dt,
)
