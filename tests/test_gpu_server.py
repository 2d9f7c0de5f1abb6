"""The continuous-batching server: same results alone, in a mix and through
the blocking calls; admission by memory budget; errors, cancel and timeouts."""
import math
import time

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_07004_gb300 import binding as B  # noqa: E402

GB = 1 << 30


@pytest.fixture(scope="module")
def mats():
    return {
        "l2d": B.Handle.from_csr(W.laplacian_2d(64, shift=0.1)),
        "l3d": B.Handle.from_csr(W.laplacian_3d(20, 18, 16, shift=0.05)),
        "mat": B.Handle.from_csr(W.matern_2d(48, 0.05)),
        "graph": B.Handle.from_csr(W.powerlaw_graph_laplacian(8000, seed=2).with_diagonal_shift(0.02)),
    }


def _same(a, b):
    assert a.logdet == b.logdet
    assert np.array_equal(a.per_probe, b.per_probe)
    assert np.array_equal(a.z_norm2, b.z_norm2)


REQS = [  # (matrix, method, probes, m, k, seed, precision)
    ("l2d", B.METHOD_OSLQ, 30, 30, 0, 0, B.FP64),
    ("l3d", B.METHOD_OSAIOP, 21, 20, 2, 1, B.FP64),
    ("mat", B.METHOD_OSLQ, 15, 25, 0, 2, B.MIXED_FP32),
    ("graph", B.METHOD_OSAIOP, 24, 18, 4, 3, B.FP64),
    ("l3d", B.METHOD_OSLQ, 30, 12, 0, 4, B.MIXED_FP32),
    ("l2d", B.METHOD_OSAIOP, 33, 15, 8, 5, B.MIXED_FP32),
    ("graph", B.METHOD_OSLQ, 24, 20, 0, 6, B.MIXED_F32X2),
    ("mat", B.METHOD_OSAIOP, 21, 16, 4, 7, B.MIXED_F32X2),
]


def _blocking(h, method, P, m, k, seed, prec):
    if method == B.METHOD_OSLQ:
        return h.oslq(P, m, seed=seed, precision=prec)
    return h.osaiop(P, m, iop_window=k, seed=seed, precision=prec)


def test_server_alone_mix_and_blocking_are_identical(mats):
    want = [_blocking(mats[r[0]], *r[1:]) for r in REQS]
    with B.Server(8 * GB, max_slots=16) as srv:
        alone = []
        for r in REQS:                                     # one at a time
            rid = srv.submit(mats[r[0]], r[1], r[2], r[3], r[4], seed=r[5], precision=r[6])
            alone.append(srv.wait(rid))
        ids = [srv.submit(mats[r[0]], r[1], r[2], r[3], r[4], seed=r[5], precision=r[6])
               for r in REQS]                              # all together
        mixed = [srv.wait(i) for i in ids]
        st = srv.stats()
    for w, a, x in zip(want, alone, mixed):
        _same(w, a)
        _same(w, x)
    assert st["completed"] == 2 * len(REQS) and st["failed"] == 0
    assert st["max_resident"] >= 2                         # requests overlapped on the GPU
    assert st["batched_steps"] > st["ticks"] / 2


def test_server_result_matches_oracle(mats):
    A = W.laplacian_2d(64, shift=0.1)
    est = O.oslq(A.to_scipy(), 30, 30, seed=0)
    with B.Server(4 * GB) as srv:
        res = srv.wait(srv.submit(mats["l2d"], B.METHOD_OSLQ, 30, 30, seed=0))
    assert abs(res.logdet - est.logdet) / abs(est.logdet) <= 1e-10
    assert res.latency_ms > 0 and res.queue_ms >= 0


def test_admission_by_memory_budget(mats):
    h = mats["l3d"]
    one = None
    with B.Server(8 * GB) as srv:
        one = srv.wait(srv.submit(h, B.METHOD_OSLQ, 30, 12, seed=9))
    # A budget that holds only one such request at a time: all still complete.
    need = h.estimate_bytes(B.METHOD_OSLQ, 30, 12)
    assert need > 0
    with B.Server(int(1.5 * need), max_slots=8) as srv:
        ids = [srv.submit(h, B.METHOD_OSLQ, 30, 12, seed=9) for _ in range(5)]
        res = [srv.wait(i, 120_000_000) for i in ids]
        st = srv.stats()
    for r in res:
        _same(one, r)
    assert st["max_resident"] == 1
    assert st["completed"] == 5


def test_request_larger_than_budget_is_rejected(mats):
    with B.Server(1 << 20) as srv:
        with pytest.raises(B.LogdetError) as e:
            srv.submit(mats["l3d"], B.METHOD_OSLQ, 30, 12)
        assert e.value.code == B.ENOMEM


def test_unknown_id_cancel_and_timeout(mats):
    with B.Server(8 * GB, max_slots=1) as srv:
        with pytest.raises(B.LogdetError) as e:
            srv.poll(987654)
        assert e.value.code == B.ENOENT
        big = srv.submit(mats["graph"], B.METHOD_OSAIOP, 60, 60, 8, seed=1)
        queued = srv.submit(mats["l2d"], B.METHOD_OSLQ, 30, 30, seed=1)
        srv.cancel(queued)
        with pytest.raises(B.LogdetError) as e:
            srv.wait(big, 0)                          # still running after 0 us
        assert e.value.code == B.ETIMEOUT
        assert srv.wait(big).logdet != 0.0
        with pytest.raises(B.LogdetError) as e:
            srv.wait(queued)
        assert e.value.code == B.ECANCEL
        with pytest.raises(B.LogdetError) as e:
            srv.submit(mats["l2d"], B.METHOD_OSLQ, 2, 5)
        assert e.value.code == B.EINVAL


def test_diagonal_shift_matches_oracle_on_shifted_matrix(mats):
    A = W.laplacian_2d(64, shift=0.1)
    sigma = 0.37
    As = A.with_diagonal_shift(sigma).to_scipy()
    for method in ("oslq", "osaiop"):
        est = O.oslq(As, 21, 20, seed=3) if method == "oslq" else O.osaiop(As, 21, 20, k=2, seed=3)
        h = mats["l2d"]
        res = h.oslq(21, 20, seed=3, shift=sigma) if method == "oslq" else \
            h.osaiop(21, 20, iop_window=2, seed=3, shift=sigma)
        assert abs(res.logdet - est.logdet) / abs(est.logdet) <= 1e-10, method
