"""The synthetic inputs: structure, sizes and analytic log-determinants."""
import numpy as np
import pytest

import workloads as W


def _check_csr(A):
    assert A.rowptr.dtype == np.int32 and A.colind.dtype == np.int32
    assert A.rowptr[0] == 0 and np.all(np.diff(A.rowptr) >= 1)
    S = A.to_scipy()
    assert abs(S - S.T).max() == 0.0
    for i in range(0, A.n, max(1, A.n // 97)):
        cols = A.colind[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0)
        assert i in cols


def test_sizes_of_the_named_workloads():
    A = W.laplacian_2d(64, shift=0.1)
    assert (A.n, A.nnz) == (4096, 20224)
    B = W.laplacian_3d(128, shift=0.01)
    assert (B.n, B.nnz) == (2097152, 14581760)
    _check_csr(A)


@pytest.mark.parametrize("maker,closed", [
    (lambda: W.laplacian_2d(9, 7, shift=0.3), lambda: W.closed_form_logdet_laplacian_2d(9, 7, 0.3)),
    (lambda: W.laplacian_3d(5, 4, 6, shift=0.02), lambda: W.closed_form_logdet_laplacian_3d(5, 4, 6, 0.02)),
    (lambda: W.matern_2d(9, 0.05), lambda: W.closed_form_logdet_matern_2d(9, 0.05)),
])
def test_closed_forms_match_dense(maker, closed):
    A = maker()
    _check_csr(A)
    dense = np.linalg.slogdet(A.to_scipy().toarray())
    assert dense[0] > 0
    assert dense[1] == pytest.approx(closed(), rel=1e-12)


def test_laplacian_3d_matches_kronecker_form():
    import scipy.sparse as sp
    N = 6
    L1 = sp.diags([-np.ones(N - 1), 2 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1])
    I = sp.eye(N)
    K = sp.kron(sp.kron(I, I), L1) + sp.kron(sp.kron(I, L1), I) + sp.kron(sp.kron(L1, I), I)
    A = W.laplacian_3d(N, shift=0.0)
    assert abs(A.to_scipy() - K).max() == 0.0


def test_matern_stencil_is_13_point():
    A = W.matern_2d(16, 0.05)
    counts = np.diff(A.rowptr)
    assert counts.max() == 13
    mid = 8 * 16 + 8
    assert counts[mid] == 13


def test_powerlaw_graph():
    G = W.powerlaw_graph_laplacian(20000, seed=3)
    _check_csr(G)
    S = G.to_scipy()
    assert np.allclose(S @ np.ones(G.n), 0.0)          # Laplacian rows sum to zero
    deg = np.diff(G.rowptr) - 1
    assert 5.0 < deg.mean() < 9.0                      # mean degree ~8 after merging
    assert deg.max() > 20 * deg.mean()                 # heavy tail
    G2 = W.powerlaw_graph_laplacian(20000, seed=3)
    assert np.array_equal(G.colind, G2.colind)         # seeded


def test_diagonal_shift():
    A = W.laplacian_2d(5).with_diagonal_shift(0.5)
    assert np.allclose(A.to_scipy().diagonal(), 4.5)


def test_graph_laplacian_from_edges():
    import scipy.sparse as sp
    edges = np.array([[0, 1], [1, 2], [2, 0], [3, 0], [0, 1], [2, 2]])  # duplicate and self-loop
    A = W.graph_laplacian(5, edges, shift=0.5)
    L = A.to_scipy().toarray()
    assert np.array_equal(L, L.T)
    np.testing.assert_allclose(L.sum(axis=1), 0.5)        # rows of D - A sum to zero
    assert L[0, 0] == 3.5 and L[4, 4] == 0.5 and L[0, 1] == -1.0
    assert np.all(np.diff(A.rowptr) >= 1)                  # every diagonal entry stored
    assert sp.csr_matrix(L).nnz == 5 + 2 * 4


def test_wendland_table_and_grid_operator():
    r = np.array([0.0, 0.25, 0.5, 0.999, 1.0, 2.0])
    phi = W.wendland_c2(r)
    assert phi[0] == 1.0 and phi[4] == 0.0 and phi[5] == 0.0
    assert np.all(np.diff(phi) <= 0)
    assert phi[1] == pytest.approx(0.75 ** 4 * 2.0)
    T = W.wendland_table(4.0, nugget=0.1)
    assert T.shape == (4, 4)                      # offsets 0..3 inside radius 4
    assert T[0, 0] == pytest.approx(1.1) and T[0, 3] > 0 and np.all(T == T.T)
    A = W.grid_operator_csr(7, 5, T)
    Q = A.to_scipy().toarray()
    assert np.array_equal(Q, Q.T)
    # entry of points (y=2, x=3) and (y=3, x=1): offsets (1, 2)
    assert Q[2 * 7 + 3, 3 * 7 + 1] == T[1, 2]
    assert np.all(np.linalg.eigvalsh(Q) > 0)      # Wendland C^2 is PD in 2D
    nnz = sum((5 - abs(dy)) * (7 - abs(dx)) for dy in range(-3, 4) for dx in range(-3, 4)
              if T[abs(dy), abs(dx)] != 0)
    assert A.nnz == nnz


def test_grf_sample_covariance():
    # covariance of the embedded field: sample variance of many fields close to
    # the diagonal of Q^{-1} (precision=True) or of Q (precision=False)
    T = W.wendland_table(3.0, nugget=0.5)
    A = W.grid_operator_csr(12, 10, T).to_scipy().toarray()
    xs = np.stack([W.grf_sample(12, 10, T, seed=s, precision=False) for s in range(4000)])
    assert abs(xs.var(axis=0).mean() / A.diagonal().mean() - 1.0) < 0.05
    xp = np.stack([W.grf_sample(12, 10, T, seed=s) for s in range(4000)])
    centre = 5 * 12 + 6
    assert abs(xp[:, centre].var() / np.linalg.inv(A)[centre, centre] - 1.0) < 0.15


def test_grf_client_table_matches_generator():
    # the GRF client builds its own tables; they must equal the generator's
    grf = pytest.importorskip("paper_2606_07004_gb300.grf")  # needs the built library
    for theta, nug in ((3.0, 0.0), (20.0, 0.1), (7.5, 0.3)):
        assert np.array_equal(grf.wendland_table(theta, nug), W.wendland_table(theta, nug))


def _csr_equal(a, b):
    return (np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.colind, b.colind)
            and np.array_equal(a.vals, b.vals) and a.vals.dtype == b.vals.dtype)


@pytest.mark.parametrize("nx,ny,shift", [(6, 2, 0.1), (7, 9, 0.0), (64, 64, 0.1), (40, 37, 0.05),
                                         (151, 149, 0.3)])
def test_laplacian_2d_direct_equals_kronecker_form(nx, ny, shift):
    # The direct stencil construction gives the same CSR (indices and doubles)
    # as kron(I, T) + kron(T, I) + shift I, T = tridiag(-1, 2, -1).
    import scipy.sparse as sp
    from workloads.matrices import _from_scipy, _lap1d
    L = sp.kron(sp.eye(ny), _lap1d(nx)) + sp.kron(_lap1d(ny), sp.eye(nx)) + shift * sp.eye(nx * ny)
    assert _csr_equal(W.laplacian_2d(nx, ny, shift), _from_scipy(L))


@pytest.mark.parametrize("N,k2", [(5, 0.05), (6, 0.05), (13, 0.3), (64, 0.05)])
def test_matern_direct_equals_sparse_product(N, k2):
    # Q = M M, M = k2 I + L_2D, formed by a sparse matrix product.
    import scipy.sparse as sp
    from workloads.matrices import _from_scipy, _lap1d
    M = sp.csr_matrix(sp.kron(sp.eye(N), _lap1d(N)) + sp.kron(_lap1d(N), sp.eye(N)) + k2 * sp.eye(N * N))
    assert _csr_equal(W.matern_2d(N, k2), _from_scipy(M @ M))
    a = W.matern_2d(N, k2, dtype=np.float32)
    assert a.vals.dtype == np.float32 and np.array_equal(a.vals, _from_scipy(M @ M).vals.astype(np.float32))
