"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This package builds sparse SPD matrices in CSR form (int32 indices, sorted
columns, explicit diagonal) and request streams.  It holds none of the
estimators' arithmetic: no probes, no Krylov steps, no logarithms of the
operator.  Both the FP64 CPU oracle and the CUDA path consume what it makes.
"""
from .matrices import (  # noqa: F401
    CSR,
    laplacian_2d,
    laplacian_3d,
    matern_2d,
    powerlaw_graph_laplacian,
    grid_stencil_3d,
    graph_laplacian,
    wendland_c2,
    wendland_table,
    grid_operator_csr,
    grf_sample,
    diagonal_matrix,
    scaled_identity,
    random_spd_dense_csr,
    permute_symmetric,
    closed_form_logdet_laplacian_2d,
    closed_form_logdet_laplacian_3d,
    closed_form_logdet_matern_2d,
)
