"""Sweep paths of the FP32 SpMM pass: x staged by TMA copies in a ring of
shared-memory windows, 2A + 1 grid lines (2D stencils) or planes (3D
stencils) at a time.  A handle created from host arrays of a grid stencil
takes the sweep for mixed-FP32 solves; a handle over device arrays of the
same matrix keeps the CSR gathers.  y is the same FP32 sum on both paths;
the window dots are reduced per sweep unit instead of per CSR tile, so the
two agree to the rounding of compensated partial sums, far inside the
mixed-precision budget (1e-4 against FP64)."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_07004_gb300 import binding as B  # noqa: E402

RTOL_PATHS = 1e-6   # sweep vs CSR gathers, both mixed FP32
RTOL_MIXED = 1e-4   # mixed vs the FP64 oracle


def _device_handle(A):
    rp = torch.as_tensor(A.rowptr.astype(np.int32), device="cuda")
    ci = torch.as_tensor(A.colind.astype(np.int32), device="cuda")
    va = torch.as_tensor(np.asarray(A.vals), device="cuda")
    return B.Handle(A.n, rp, ci, va, device=True)


def _csr(Q, dtype=np.float32):
    Q = Q.tocsr()
    Q.sort_indices()
    return W.CSR(Q.shape[0], Q.indptr.astype(np.int32), Q.indices.astype(np.int32),
                 Q.data.astype(dtype))


def _band(L, n, dtype=np.float32):
    # 5-diagonal SPD band (offsets 0, +-1, +-L) whose last line is ragged
    # (n not a multiple of L).
    return _csr(sp.diags([np.full(n - L, -1.0), np.full(n - 1, -1.0), np.full(n, 4.2),
                          np.full(n - 1, -1.0), np.full(n - L, -1.0)], [-L, -1, 0, 1, L]), dtype)


def _band3(nx, ny, nz):
    # The 3D Laplacian's 7 offsets as full bands: entries wrap across line and
    # plane edges, so the matrix is no grid stencil.
    n = nx * ny * nz
    offs = [-nx * ny, -nx, -1, 0, 1, nx, nx * ny]
    return _csr(sp.diags([np.full(n - abs(o), 6.5 if o == 0 else -1.0) for o in offs], offs))


FACES = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]

MATS = {
    "lap2d": (lambda: W.laplacian_2d(100, 90, shift=0.05), (2, 100, 1)),
    "matern": (lambda: W.matern_2d(70, 0.05, dtype=np.float32), (2, 70, 2)),
    "band-ragged": (lambda: _band(64, 5001), (2, 64, 1)),
    "lap3d": (lambda: W.laplacian_3d(24, 21, 19, shift=0.01), (3, 24, 1)),
    "lap3d-thin": (lambda: W.laplacian_3d(37, 5, 40, shift=0.02, dtype=np.float32), (3, 37, 1)),
    # wider 3D stencils: |dx|, |dy| <= 2 (halo of two points), |dz| <= 2 (ring of 5 planes)
    "grid3-wide": (lambda: W.grid_stencil_3d(20, 15, 30, FACES + [(2, 0, 0), (-2, 0, 0),
                                                                   (0, 2, 0), (0, -2, 0)]),
                   (3, 20, 1)),
    "grid3-deep": (lambda: W.grid_stencil_3d(16, 16, 20, FACES + [(0, 0, 2), (0, 0, -2)]),
                   (3, 16, 2)),
}


def _close(a, b, rtol=RTOL_PATHS):
    assert abs(a.logdet - b.logdet) <= rtol * abs(b.logdet)
    scale = np.max(np.abs(b.per_probe))
    np.testing.assert_allclose(a.per_probe, b.per_probe, rtol=0, atol=10 * rtol * scale)


def _same(a, b):
    assert a.logdet == b.logdet
    assert np.array_equal(a.per_probe, b.per_probe)
    assert np.array_equal(a.z_norm2, b.z_norm2)


def test_grid_structure_detection():
    for name, (mk, want) in MATS.items():
        A = mk()
        with B.Handle.from_csr(A) as h, _device_handle(A) as hd:
            assert h.grid_structure() == want, name
            assert hd.grid_structure() == (0, 0, 0)
    for A in (W.laplacian_2d(40, 40, shift=0.1), _band3(24, 21, 19)):
        with B.Handle.from_csr(A) as h:   # n < 4096; bands that wrap
            assert h.grid_structure() == (0, 0, 0)


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("method,k", [("oslq", 0), ("osaiop", 2), ("osaiop", 4), ("osaiop", 8)])
def test_sweep_matches_csr_path(name, method, k):
    A = MATS[name][0]()
    with B.Handle.from_csr(A) as hs, _device_handle(A) as hc:
        for kw in ({}, {"shift": 0.02}, {"autotune": 1}):
            if method == "oslq":
                a = hs.oslq(36, 20, seed=3, precision=B.MIXED_FP32, **kw)
                b = hc.oslq(36, 20, seed=3, precision=B.MIXED_FP32, **kw)
            else:
                a = hs.osaiop(36, 16, iop_window=k, seed=3, precision=B.MIXED_FP32, **kw)
                b = hc.osaiop(36, 16, iop_window=k, seed=3, precision=B.MIXED_FP32, **kw)
            _close(a, b)


@pytest.mark.parametrize("name", ["matern", "band-ragged", "lap3d", "lap3d-thin", "grid3-wide",
                                  "grid3-deep"])
def test_sweep_against_fp64_oracle(name):
    A = MATS[name][0]()
    Q = A.to_scipy()
    with B.Handle.from_csr(A) as h:
        r1 = h.oslq(30, 25, seed=2, precision=B.MIXED_FP32)
        r2 = h.osaiop(30, 20, iop_window=4, seed=2, precision=B.MIXED_FP32)
    e1 = O.oslq(Q, 30, 25, seed=2)
    e2 = O.osaiop(Q, 30, 20, k=4, seed=2)
    assert abs(r1.logdet - e1.logdet) <= RTOL_MIXED * abs(e1.logdet)
    assert abs(r2.logdet - e2.logdet) <= RTOL_MIXED * abs(e2.logdet)


def test_sweep_wide_block_deterministic_server_and_plan():
    # 120 probes (80-column Krylov block); repeated runs, the server and a
    # graph plan take the same launches and give bit-identical results.
    A = W.matern_2d(90, 0.05, dtype=np.float32)
    with B.Handle.from_csr(A) as hs, _device_handle(A) as hc:
        a = hs.oslq(120, 12, seed=1, precision=B.MIXED_FP32)
        _same(a, hs.oslq(120, 12, seed=1, precision=B.MIXED_FP32))
        _close(a, hc.oslq(120, 12, seed=1, precision=B.MIXED_FP32))
        with B.Server(8 << 30) as srv:
            ids = [srv.submit(hs, B.METHOD_OSAIOP, 30, 12, 4, seed=s, precision=B.MIXED_FP32)
                   for s in range(3)]
            served = [srv.wait(i) for i in ids]
        with B.Plan(hs, B.METHOD_OSAIOP, 30, 12, 4, precision=B.MIXED_FP32) as plan:
            replay = [plan.run(s) for s in range(3)]
        for s in range(3):
            want = hs.osaiop(30, 12, iop_window=4, seed=s, precision=B.MIXED_FP32)
            _same(served[s], want)
            _same(replay[s], want)


def test_sweep_mixed_batch_in_server():
    # One server batch holds line-sweep jobs of different stencils (5 and 13
    # diagonals, A = 1 and 2, one ragged last line), a plane-sweep job (3D
    # stencil), a CSR job (wrapping bands) and both methods: the launch takes
    # the generic diagonal-count instance and the largest ring, and splits
    # by path.  Each result must equal the same request alone.
    mats = [W.laplacian_2d(100, 90, shift=0.05), W.matern_2d(70, 0.05, dtype=np.float32),
            _band(64, 5001), W.laplacian_3d(24, 21, 19, shift=0.01), _band3(24, 21, 19)]
    hs = [B.Handle.from_csr(A) for A in mats]
    try:
        reqs = []
        for i, h in enumerate(hs):
            reqs.append((h, B.METHOD_OSLQ, 0, i, 0.0))
            reqs.append((h, B.METHOD_OSAIOP, 4, 10 + i, 0.02))
        with B.Server(8 << 30) as srv:
            ids = [srv.submit(h, meth, 30, 12, k, seed=sd, precision=B.MIXED_FP32, shift=sh)
                   for h, meth, k, sd, sh in reqs]
            got = [srv.wait(i) for i in ids]
        for (h, meth, k, sd, sh), g in zip(reqs, got):
            if meth == B.METHOD_OSLQ:
                want = h.oslq(30, 12, seed=sd, precision=B.MIXED_FP32, shift=sh)
            else:
                want = h.osaiop(30, 12, iop_window=k, seed=sd, precision=B.MIXED_FP32, shift=sh)
            _same(g, want)
    finally:
        for h in hs:
            h.close()


def test_sweep_wait_timeout_reports_and_recovers(monkeypatch):
    # LOGDET_TEST_SWEEP_STALL=1 arms each ring barrier for 16 bytes more than
    # its copies deliver: every bounded wait runs out (20 ms), the CTAs wait
    # for their copies, flag the job and return.  The solve must fail with
    # LOGDET_ETIMEOUT and the next solve on the same handle must be exact.
    A = W.laplacian_2d(100, 90, shift=0.05)
    with B.Handle.from_csr(A) as h:
        want = h.oslq(30, 6, seed=1, precision=B.MIXED_FP32)
        monkeypatch.setenv("LOGDET_TEST_SWEEP_STALL", "1")
        with pytest.raises(B.LogdetError) as e:
            h.oslq(30, 6, seed=1, precision=B.MIXED_FP32)
        assert e.value.code == B.ETIMEOUT
        monkeypatch.delenv("LOGDET_TEST_SWEEP_STALL")
        _same(h.oslq(30, 6, seed=1, precision=B.MIXED_FP32), want)


def test_memory_estimate_counts_sweep_values():
    # Admission by memory: an FP32 solve of a grid stencil also holds the
    # values per row and diagonal (16 floats per row for 13 diagonals).
    A = W.matern_2d(90, 0.05, dtype=np.float32)
    with B.Handle.from_csr(A) as hs, _device_handle(A) as hc:
        a = hs.estimate_bytes(B.METHOD_OSLQ, 30, 12, precision=B.MIXED_FP32)
        b = hc.estimate_bytes(B.METHOD_OSLQ, 30, 12, precision=B.MIXED_FP32)
        assert a - b == 16 * A.n * 4
        assert hs.estimate_bytes(B.METHOD_OSLQ, 30, 12) == hc.estimate_bytes(B.METHOD_OSLQ, 30, 12)
