"""Grid-structure detection of the sweep paths (host code, no GPU): which
stencils take the line sweep (dim 2: offsets l L + c) or the plane sweep
(dim 3: an L x ny x nz grid stencil with no entry wrapping across an edge),
with the line stride and reach the kernels are built around."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W

B = pytest.importorskip("paper_2606_07004_gb300.binding")


def _csr(Q):
    Q = Q.tocsr()
    Q.sort_indices()
    return W.CSR(Q.shape[0], Q.indptr.astype(np.int32), Q.indices.astype(np.int32),
                 Q.data.astype(np.float64))


def _bands(n, offs, diag=8.0):
    return _csr(sp.diags([np.full(n - abs(o), diag if o == 0 else -1.0) for o in offs], offs))


def _grid3(nx, ny, nz, taps):
    return W.grid_stencil_3d(nx, ny, nz, taps)


FACES = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]


@pytest.mark.parametrize("A,want", [
    (W.laplacian_2d(100, 90), (2, 100, 1)),
    (W.laplacian_2d(64, 70), (2, 64, 1)),
    (W.matern_2d(70, 0.05), (2, 70, 2)),
    (W.matern_2d(1024, 0.05), (2, 1024, 2)),
    (_bands(5001, [-64, -1, 0, 1, 64]), (2, 64, 1)),          # ragged last line
    (_bands(8000, [-300, -3, 0, 3, 300]), (2, 300, 1)),
    (W.laplacian_3d(24, 21, 19), (3, 24, 1)),
    (W.laplacian_3d(37, 5, 40), (3, 37, 1)),
    (W.laplacian_3d(20, 20, 30), (3, 20, 1)),   # half the plane also splits, but wraps
    (W.laplacian_3d(100), (3, 100, 1)),
    (_grid3(20, 15, 30, FACES + [(2, 0, 0), (-2, 0, 0), (0, 2, 0), (0, -2, 0)]), (3, 20, 1)),
    (_grid3(16, 16, 20, FACES + [(0, 0, 2), (0, 0, -2)]), (3, 16, 2)),
])
def test_detected_structure(A, want):
    assert B.grid_structure_csr(A) == want


@pytest.mark.parametrize("A", [
    W.laplacian_2d(40, 40),                                   # n < 4096
    _bands(9576, [-504, -24, -1, 0, 1, 24, 504]),             # 3D offsets, entries wrap edges
    _grid3(12, 12, 40, FACES + [(0, 3, 0), (0, -3, 0)]),      # |dy| = 3
    _bands(9000, list(range(-8, 9)) + [-40, 40]),             # 19 diagonals > 16
    W.powerlaw_graph_laplacian(5000, seed=3),                 # unstructured
])
def test_no_structure(A):
    assert B.grid_structure_csr(A) == (0, 0, 0)


def test_invalid_arguments():
    with pytest.raises(B.LogdetError):
        B.grid_structure_csr(W.CSR(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0)))
