"""Synthetic sparse SPD matrices in CSR form.

Every generator returns a :class:`CSR` with int32 ``rowptr``/``colind``,
columns sorted within each row, no duplicates and an explicit diagonal entry
in every row.  Grid operators use lexicographic ordering with x fastest and
Dirichlet boundaries; the stencils are the unscaled integer ones (2D: 4 on the
diagonal, -1 to each neighbour; 3D: 6 and -1).

These stand in for the paper's sparse test matrices (Sec. 4, Table 1), which
are not shipped: shifted 2D/3D Laplacians (structured FEM/FD-like operators),
an SPDE-style Matern precision ``(kappa^2 I + L)^2`` (the GRF workload of
Sec. 4), and a Chung-Lu power-law graph Laplacian (irregular sparsity).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class CSR:
    """A square sparse matrix in compressed-sparse-row form (host arrays)."""

    n: int
    rowptr: np.ndarray  # int32, n+1
    colind: np.ndarray  # int32, nnz
    vals: np.ndarray    # float64 or float32, nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self, dtype=np.float64) -> sp.csr_matrix:
        return sp.csr_matrix(
            (self.vals.astype(dtype, copy=False), self.colind, self.rowptr),
            shape=(self.n, self.n),
        )

    def astype(self, dtype) -> "CSR":
        return CSR(self.n, self.rowptr, self.colind, self.vals.astype(dtype))

    def with_diagonal_shift(self, shift: float) -> "CSR":
        """Return Q + shift*I (diagonal entries are present by construction)."""
        vals = self.vals.copy()
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.rowptr))
        diag = self.colind.astype(np.int64) == rows
        vals[diag] += vals.dtype.type(shift)
        return CSR(self.n, self.rowptr, self.colind, vals)


def _from_scipy(A: sp.spmatrix, dtype=np.float64) -> CSR:
    A = sp.csr_matrix(A)
    A.sum_duplicates()
    A.sort_indices()
    n = A.shape[0]
    # Make sure every diagonal entry is stored (explicit zero if absent).
    d = A.diagonal()
    missing = np.flatnonzero(np.asarray(
        (A != 0).multiply(sp.eye(n, format="csr")).sum(axis=1)).ravel() == 0)
    if missing.size:
        A = A + sp.csr_matrix((np.zeros(missing.size), (missing, missing)), shape=(n, n))
        A = sp.csr_matrix(A)
        A.sort_indices()
    del d
    if A.nnz >= 2**31:
        raise ValueError("nnz does not fit int32 CSR indices")
    return CSR(
        n,
        A.indptr.astype(np.int32),
        A.indices.astype(np.int32),
        A.data.astype(dtype),
    )


def graph_laplacian(n: int, edges: np.ndarray, shift: float = 0.0, dtype=np.float64) -> CSR:
    """L = D - A + shift*I of the undirected graph on n nodes with unit-weight
    edges (an (E, 2) array of node pairs; self-loops dropped, duplicates merged)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    Adj = sp.csr_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n))
    Adj = ((Adj + Adj.T) > 0).astype(np.float64)
    deg = np.asarray(Adj.sum(axis=1)).ravel()
    return _from_scipy(sp.diags(deg + shift) - Adj, dtype)


def wendland_c2(r: np.ndarray) -> np.ndarray:
    """Wendland's C^2 function for d <= 3: (1 - r)^4 (4 r + 1) on [0, 1), 0 beyond."""
    r = np.asarray(r, dtype=np.float64)
    return np.where(r < 1.0, (1.0 - r) ** 4 * (4.0 * r + 1.0), 0.0)


def wendland_table(theta: float, nugget: float = 0.0) -> np.ndarray:
    """Quadrant table W[|dy|, |dx|] = phi(sqrt(dx^2 + dy^2) / theta) of the
    Wendland C^2 covariance with support radius theta grid cells, plus a
    nugget on W[0, 0]; (R + 1) x (R + 1) with R the largest offset inside the
    support."""
    R = max(0, int(math.ceil(theta)) - 1)
    d = np.hypot(*np.meshgrid(np.arange(R + 1), np.arange(R + 1), indexing="ij"))
    W = wendland_c2(d / theta)
    W[0, 0] += nugget
    return W


def grid_operator_csr(nx: int, ny: int, W: np.ndarray, dtype=np.float64) -> CSR:
    """Explicit CSR of the gridded operator Q[(y,x),(y',x')] = W[|y-y'|, |x-x'|]
    (row index y * nx + x), for grids small enough to store."""
    R = W.shape[0] - 1
    rows, cols, vals = [], [], []
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            w = W[abs(dy), abs(dx)]
            if w == 0.0:
                continue
            ok = (yy + dy >= 0) & (yy + dy < ny) & (xx + dx >= 0) & (xx + dx < nx)
            r = (yy * nx + xx)[ok]
            rows.append(r)
            cols.append(r + dy * nx + dx)
            vals.append(np.full(r.size, w))
    n = nx * ny
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    return _from_scipy(A, dtype)


def grf_sample(nx: int, ny: int, W: np.ndarray, seed: int, precision: bool = True) -> np.ndarray:
    """A seeded Gaussian random field on the nx x ny grid (row-major, y * nx + x)
    by circulant embedding of the gridded operator W on a periodic grid of at
    least (ny + R) x (nx + R) points: precision=True draws from N(0, Q^{-1})
    (Q the embedded operator), else from N(0, Q).  Raises if the embedding is
    not positive definite."""
    R = W.shape[0] - 1
    My, Mx = ny + R + 1, nx + R + 1
    c = np.zeros((My, Mx))
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            c[dy % My, dx % Mx] += W[abs(dy), abs(dx)]
    lam = np.real(np.fft.fft2(c))
    if lam.min() <= 0:
        raise ValueError("circulant embedding is not positive definite")
    spec = 1.0 / lam if precision else lam
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((My, Mx)) + 1j * rng.standard_normal((My, Mx))
    f = np.fft.fft2(np.sqrt(spec / (My * Mx)) * z)
    return np.ascontiguousarray(np.real(f)[:ny, :nx]).ravel()


def _lap1d(N: int) -> sp.csr_matrix:
    return sp.diags([-np.ones(N - 1), 2 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1], format="csr")


def _grid_stencil_csr(nx: int, ny: int, taps, dtype) -> CSR:
    """CSR of a 2D stencil on an nx x ny grid (row y nx + x), built directly.

    taps: (dx, dy, value) in ascending column order (dy nx + dx); value is a
    scalar or a per-row array.  A tap is stored for a row when its neighbour
    lies in the grid (no wrapping across grid edges)."""
    n = nx * ny
    T = len(taps)
    x = np.tile(np.arange(nx, dtype=np.int32), ny)
    y = np.repeat(np.arange(ny, dtype=np.int32), nx)
    # n x T tables in row-major order: a row's stored taps come out in tap
    # (= ascending column) order when the valid ones are selected.
    valid = np.empty((n, T), dtype=bool)
    cols = np.empty((n, T), dtype=np.int32)
    vals = np.empty((n, T), dtype=np.float64)
    rows = np.arange(n, dtype=np.int32)
    for t, (dx, dy, val) in enumerate(taps):
        valid[:, t] = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny)
        cols[:, t] = rows + (dy * nx + dx)
        vals[:, t] = val
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(valid.sum(axis=1), out=rowptr[1:])
    return CSR(n, rowptr.astype(np.int32), cols[valid], vals[valid].astype(dtype, copy=False))


def laplacian_2d(nx: int, ny: int | None = None, shift: float = 0.0, dtype=np.float64) -> CSR:
    """5-point Dirichlet Laplacian on an nx x ny grid, plus shift*I (diagonal
    4 + shift, neighbours -1; built directly, the same doubles as
    kron(I, T) + kron(T, I) + shift I with T = tridiag(-1, 2, -1))."""
    ny = nx if ny is None else ny
    if nx < 6 or ny < 2:   # small grids: the Kronecker form (it also stores some zeros)
        L = sp.kron(sp.eye(ny), _lap1d(nx)) + sp.kron(_lap1d(ny), sp.eye(nx))
        return _from_scipy(L + shift * sp.eye(nx * ny), dtype)
    d = 4.0 + shift
    taps = [(0, -1, -1.0), (-1, 0, -1.0), (0, 0, d), (1, 0, -1.0), (0, 1, -1.0)]
    return _grid_stencil_csr(nx, ny, taps, dtype)


def laplacian_3d(nx: int, ny: int | None = None, nz: int | None = None,
                 shift: float = 0.0, dtype=np.float64) -> CSR:
    """7-point Dirichlet Laplacian on an nx x ny x nz grid, plus shift*I.

    Built directly (not through Kronecker products) so that the 2M-row case
    is produced in about a second.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    # Column offsets in sorted order: -nx*ny, -nx, -1, 0, +1, +nx, +nx*ny.
    offs = [-nx * ny, -nx, -1, 0, 1, nx, nx * ny]
    valid = [z > 0, y > 0, x > 0, np.ones(n, bool), x < nx - 1, y < ny - 1, z < nz - 1]
    counts = np.zeros(n, dtype=np.int64)
    for v in valid:
        counts += v
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    colind = np.empty(nnz, dtype=np.int32)
    vals = np.empty(nnz, dtype=np.float64)
    pos = rowptr[:-1].copy()
    diag_val = 6.0 + shift
    for off, v in zip(offs, valid):
        rows = idx[v]
        p = pos[v]
        colind[p] = (rows + off).astype(np.int32)
        vals[p] = diag_val if off == 0 else -1.0
        pos[v] += 1
    return CSR(n, rowptr.astype(np.int32), colind, vals.astype(dtype))


def matern_2d(N: int, kappa2: float, dtype=np.float64) -> CSR:
    """SPDE-style Matern precision Q = M @ M with M = kappa2*I + L_2D (N x N grid).

    In the interior this is the 13-point stencil.  Entry (i, j) of M M sums
    M_ik M_kj over the paths i -> k -> j of the grid: c^2 plus one per
    in-grid neighbour on the diagonal (c = 4 + kappa2, the neighbours added in
    column order around c^2, as a sparse product forms it), -2c for a
    neighbour, 1 for a point two steps away in a line and 2 for a diagonal
    neighbour.  Built directly in FP64 and cast at the end.
    """
    if N < 5:
        M = sp.kron(sp.eye(N), _lap1d(N)) + sp.kron(_lap1d(N), sp.eye(N)) + kappa2 * sp.eye(N * N)
        M = sp.csr_matrix(M)
        return _from_scipy(M @ M, dtype)
    c = (2.0 + 2.0) + kappa2
    idx = np.arange(N * N, dtype=np.int64)
    x, y = idx % N, idx // N
    diag = np.zeros(N * N)
    diag += (y > 0)
    diag += (x > 0)
    diag += c * c
    diag += (x < N - 1)
    diag += (y < N - 1)
    e = -c + -c
    taps = [(0, -2, 1.0), (-1, -1, 2.0), (0, -1, e), (1, -1, 2.0),
            (-2, 0, 1.0), (-1, 0, e), (0, 0, diag), (1, 0, e), (2, 0, 1.0),
            (-1, 1, 2.0), (0, 1, e), (1, 1, 2.0), (0, 2, 1.0)]
    return _grid_stencil_csr(N, N, taps, dtype)


def grid_stencil_3d(nx: int, ny: int, nz: int, taps, diag: float = 30.0,
                    dtype=np.float64) -> CSR:
    """A 3D stencil on an nx x ny x nz grid (row (z ny + y) nx + x): diag on
    the diagonal and -1 for each (dx, dy, dz) tap whose neighbour lies in the
    grid (no wrapping across edges).  Diagonally dominant (SPD) when diag
    exceeds the number of taps."""
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    x, y, z = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    rows, cols = [idx], [idx]
    for dx, dy, dz in taps:
        ok = ((x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny)
              & (z + dz >= 0) & (z + dz < nz))
        rows.append(idx[ok])
        cols.append(idx[ok] + dx + dy * nx + dz * nx * ny)
    r, c = np.concatenate(rows), np.concatenate(cols)
    v = np.where(r == c, diag, -1.0)
    return _from_scipy(sp.csr_matrix((v, (r, c)), shape=(n, n)), dtype)


def powerlaw_graph_laplacian(n: int, exponent: float = 2.3, mean_degree: float = 8.0,
                             seed: int = 0, dtype=np.float64) -> CSR:
    """Chung-Lu random graph Laplacian L = D - A (unit weights, no self loops).

    Expected degrees follow w_i proportional to (i + i0)^(-1/(exponent-1)),
    scaled to the requested mean; i0 is chosen so the largest expected degree
    is sqrt(n * mean_degree), the usual Chung-Lu admissibility cap.  Edges are
    drawn as n*mean/2 independent endpoint pairs with probability w_i/sum(w);
    duplicates are merged and self loops dropped.  The result is singular
    (constant null vector): add a diagonal shift before use.
    """
    rng = np.random.default_rng(seed)
    g = 1.0 / (exponent - 1.0)
    target_max = math.sqrt(n * mean_degree)
    i = np.arange(n, dtype=np.float64)

    def max_over_mean(i0):
        w = (i + i0) ** (-g)
        return w[0] / w.mean()

    lo, hi = 0.0, float(n)
    want = target_max / mean_degree
    for _ in range(100):  # max/mean decreases as i0 grows
        mid = 0.5 * (lo + hi)
        if max_over_mean(mid) > want:
            lo = mid
        else:
            hi = mid
    w = (i + hi) ** (-g)
    w *= mean_degree / w.mean()
    p = w / w.sum()
    cdf = np.cumsum(p)
    cdf[-1] = 1.0
    m_edges = int(round(n * mean_degree / 2))
    u = np.searchsorted(cdf, rng.random(m_edges), side="right").astype(np.int64)
    v = np.searchsorted(cdf, rng.random(m_edges), side="right").astype(np.int64)
    np.minimum(u, n - 1, out=u)
    np.minimum(v, n - 1, out=v)
    keep = u != v
    u, v = u[keep], v[keep]
    # Entry keys row * n + col of both triangles and the diagonal, sorted
    # (row-major CSR order), duplicates merged.
    idx = np.arange(n, dtype=np.int64)
    keys = np.concatenate([u * n + v, v * n + u, idx * (n + 1)])
    keys.sort()
    keys = keys[np.concatenate(([True], keys[1:] != keys[:-1]))]
    rows = keys // n
    cols = keys - rows * n
    diag = rows == cols
    deg = np.bincount(rows[~diag], minlength=n).astype(np.float64)
    all_vals = np.where(diag, deg[rows], -1.0)
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 CSR indices")
    return CSR(n, rowptr.astype(np.int32), cols.astype(np.int32), all_vals.astype(dtype))


def diagonal_matrix(d, dtype=np.float64) -> CSR:
    d = np.asarray(d, dtype=np.float64)
    n = d.size
    return CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d.astype(dtype))


def scaled_identity(n: int, c: float, dtype=np.float64) -> CSR:
    return diagonal_matrix(np.full(n, c), dtype)


def random_spd_dense_csr(n: int, seed: int, cond: float = 100.0, dtype=np.float64) -> CSR:
    """Dense random SPD matrix with eigenvalues log-spaced in [1, cond], stored as CSR."""
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.logspace(0.0, math.log10(cond), n)
    A = (Qm * lam) @ Qm.T
    A = 0.5 * (A + A.T)
    return _from_scipy(sp.csr_matrix(A), dtype)


def permute_symmetric(A: CSR, perm: np.ndarray) -> CSR:
    """Return P A P^T where row i of the result is row perm[i] of A."""
    S = A.to_scipy()
    P = S[perm][:, perm]
    return _from_scipy(P, A.vals.dtype)


# ---------------------------------------------------------------------------
# Closed-form log-determinants from analytic Dirichlet eigenvalues.
# ---------------------------------------------------------------------------

def _lap1d_eigs(N: int) -> np.ndarray:
    k = np.arange(1, N + 1, dtype=np.float64)
    return 2.0 - 2.0 * np.cos(k * math.pi / (N + 1))


def closed_form_logdet_laplacian_2d(nx: int, ny: int | None = None, shift: float = 0.0) -> float:
    ny = nx if ny is None else ny
    ex, ey = _lap1d_eigs(nx), _lap1d_eigs(ny)
    return float(math.fsum(np.log(ex[None, :] + ey[:, None] + shift).ravel()))


def closed_form_logdet_laplacian_3d(nx: int, ny: int | None = None, nz: int | None = None,
                                    shift: float = 0.0) -> float:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    ex, ey, ez = _lap1d_eigs(nx), _lap1d_eigs(ny), _lap1d_eigs(nz)
    total = []
    for z in ez:
        total.append(math.fsum(np.log(ex[None, :] + ey[:, None] + z + shift).ravel()))
    return float(math.fsum(total))


def closed_form_logdet_matern_2d(N: int, kappa2: float) -> float:
    e = _lap1d_eigs(N)
    mu = e[None, :] + e[:, None]
    return float(math.fsum((2.0 * np.log(kappa2 + mu)).ravel()))
