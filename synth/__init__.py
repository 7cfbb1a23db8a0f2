"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package holds only input generation: sparse SPD matrices in CSR form
(full symmetric pattern, sorted columns), right-hand sides and the small
random test matrices, and the seeded initial weights of the shift-predictor
network.  It contains none of the method's arithmetic and imports neither the
oracle nor the CUDA library.
"""
from .matrices import (  # noqa: F401
    Problem,
    poisson2d_5pt,
    laplace3d_27pt,
    diffusion3d_7pt,
    elasticity3d_q1,
    diffusion_batch,
    random_spd,
    tridiagonal_spd,
    rhs,
    config_problem,
    is_exactly_symmetric,
)
from .params import mlp_init  # noqa: F401,E402
