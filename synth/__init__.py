"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This package holds no arithmetic of the contour-integral method: it only builds
the split-form problems (constant sparse matrices A_i plus descriptions of the
scalar functions f_i, as in the split form T(z) = sum_i A_i f_i(z), Sec. 2
Eq. (split)), contour regions, and the random probe block V.
"""
from .problems import (  # noqa: F401
    Problem, delay_1d, delay_2d, drude_2d, sqrt_3d, diagonal_delay, diagonal_drude,
    diagonal_sqrt, dense_drude_small, dense_linear_small, config_problem, CONFIGS,
    random_probe_block, serving_requests, serving_problem,
)
