"""Diagonal fast path of the FP32 SpMM pass (x staged by TMA copies per band
of diagonals).  A handle created from host arrays of a stencil matrix takes
the path for mixed-FP32 solves; a handle over device arrays of the same matrix
keeps the CSR gathers.  The two must give bit-identical results: same tiles,
same row order per thread, same summation order per row."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_07004_gb300 import binding as B  # noqa: E402


def _device_handle(A):
    rp = torch.as_tensor(A.rowptr.astype(np.int32), device="cuda")
    ci = torch.as_tensor(A.colind.astype(np.int32), device="cuda")
    va = torch.as_tensor(np.asarray(A.vals), device="cuda")
    return B.Handle(A.n, rp, ci, va, device=True)


MATS = {
    "lap2d": lambda: W.laplacian_2d(100, 90, shift=0.05),
    "lap3d": lambda: W.laplacian_3d(24, 21, 19, shift=0.01),
    "matern": lambda: W.matern_2d(70, 0.05, dtype=np.float32),
}


def _same(a, b):
    assert a.logdet == b.logdet
    assert np.array_equal(a.per_probe, b.per_probe)
    assert np.array_equal(a.z_norm2, b.z_norm2)


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("method,k", [("oslq", 0), ("osaiop", 2), ("osaiop", 4), ("osaiop", 8)])
def test_diagonal_path_bit_identical_to_csr(name, method, k):
    A = MATS[name]()
    with B.Handle.from_csr(A) as hd, _device_handle(A) as hc:
        for kw in ({}, {"shift": 0.02}, {"autotune": 1}):
            if method == "oslq":
                a = hd.oslq(36, 20, seed=3, precision=B.MIXED_FP32, **kw)
                b = hc.oslq(36, 20, seed=3, precision=B.MIXED_FP32, **kw)
            else:
                a = hd.osaiop(36, 16, iop_window=k, seed=3, precision=B.MIXED_FP32, **kw)
                b = hc.osaiop(36, 16, iop_window=k, seed=3, precision=B.MIXED_FP32, **kw)
            _same(a, b)


def test_diagonal_path_wide_block_and_server():
    # 120 probes (80-column Krylov block, 5 bands of staged rows)
    A = W.matern_2d(90, 0.05, dtype=np.float32)
    with B.Handle.from_csr(A) as hd, _device_handle(A) as hc:
        a = hd.oslq(120, 12, seed=1, precision=B.MIXED_FP32)
        b = hc.oslq(120, 12, seed=1, precision=B.MIXED_FP32)
        _same(a, b)
        with B.Server(8 << 30) as srv:
            ids = [srv.submit(hd, B.METHOD_OSAIOP, 30, 12, 4, seed=s, precision=B.MIXED_FP32)
                   for s in range(3)]
            served = [srv.wait(i) for i in ids]
        for s in range(3):
            _same(served[s], hc.osaiop(30, 12, iop_window=4, seed=s, precision=B.MIXED_FP32))
