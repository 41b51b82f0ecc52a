"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package builds test problems only: finite-difference convection-diffusion
matrices in CSR form and right-hand sides.  It contains none of the solver's
arithmetic (no SpMV kernel, no orthogonalisation, no least squares), so both
the CPU oracle and the CUDA path can consume its arrays without sharing code.
"""
from .stencil import (  # noqa: F401
    Problem,
    conv_diff_2d,
    conv_diff_3d,
    random_wind,
    rhs_manufactured,
    rhs_ones,
    rhs_ones_plus_noise,
    config_small_2d,
    config_3d,
    config_aniso_2d,
    batched_systems,
    selector_matrices,
    build_selector_matrix,
    MLP_SHAPES,
    mlp_init,
    stencil_matrix,
    laplace_2d,
    laplace_3d,
    uniflow_2d,
    bentpipe_2d,
    box_2d,
    star_3d,
    box_3d,
    shuffled,
    scaled,
    config_bj,
)
