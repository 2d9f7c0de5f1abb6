"""Preemption in the serving queue (logdet_suspend / logdet_resume).

A suspended request leaves the batch at a tick boundary with every device
buffer of its solve copied to host memory and freed; resumed, it is
re-admitted at the front of the queue, gets its buffers back (at new
addresses) and continues from the step where it stopped.  The result must be
bit-identical to the uninterrupted solve (which the server already matches
bit for bit with the blocking API), the budget must be free while it is
held, and the error cases must be reported."""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_07004_gb300 import binding as B  # noqa: E402


def _same(a, b):
    assert a.logdet == b.logdet
    assert (a.tr_sub, a.tr_res, a.s_eff, a.steps_max, a.status_bits) == \
        (b.tr_sub, b.tr_res, b.s_eff, b.steps_max, b.status_bits)
    assert np.array_equal(a.per_probe, b.per_probe)


def _until(srv, key, value, timeout=30.0):
    t0 = time.time()
    while time.time() - t0 < timeout:
        if srv.stats()[key] == value:
            return True
        time.sleep(0.002)
    return False


@pytest.mark.parametrize("method,k,precision", [
    (B.METHOD_OSLQ, 0, B.FP64),
    (B.METHOD_OSAIOP, 4, B.FP64),          # phase-1 basis, window ring, Hessenberg state
    (B.METHOD_OSAIOP, 2, B.MIXED_FP32),    # line sweep of a grid stencil
    (B.METHOD_OSAIOP, 4, B.MIXED_F32X2),   # double-float blocks
])
def test_suspend_mid_krylov_resume_is_bit_identical(method, k, precision):
    A = (W.matern_2d(512, 0.05, dtype=np.float32) if precision == B.MIXED_FP32
         else W.laplacian_3d(96, shift=0.01))
    P, m = 60, 120
    with B.Handle.from_csr(A) as h:
        ref = (h.oslq(P, m, seed=4, precision=precision) if method == B.METHOD_OSLQ
               else h.osaiop(P, m, iop_window=k, seed=4, precision=precision))
        with B.Server(64 << 30, max_slots=4) as srv:
            rid = srv.submit(h, method, P, m, k, seed=4, precision=precision)
            time.sleep(0.5 * ref.device_ms / 1e3)   # about half way
            srv.suspend(rid)
            assert _until(srv, "suspended", 1) or srv.poll(rid) is not None
            st = srv.stats()
            if st["suspended"] == 1:
                assert srv.poll(rid) is None            # pending while held
                assert st["bytes_in_use"] == 0 and st["resident"] == 0
                srv.resume(rid)
            got = srv.wait(rid)
            st = srv.stats()
    _same(got, ref)
    # the suspension was taken inside a Krylov phase in this configuration
    assert st["suspensions"] == 1 and st["suspended_in_krylov"] == 1


def test_held_budget_goes_to_other_requests_and_cycles():
    A = W.laplacian_3d(64, shift=0.02)
    P, m = 30, 150
    with B.Handle.from_csr(A) as h:
        need = h.estimate_bytes(B.METHOD_OSAIOP, P, m, 4)
        ref_a = h.osaiop(P, m, iop_window=4, seed=1)
        ref_b = h.osaiop(P, m, iop_window=4, seed=2)
        # room for one request at a time
        with B.Server(int(need * 1.5), max_slots=4) as srv:
            a = srv.submit(h, B.METHOD_OSAIOP, P, m, 4, seed=1)
            b = srv.submit(h, B.METHOD_OSAIOP, P, m, 4, seed=2)
            for cycle in range(3):          # suspend and resume a, three times
                time.sleep(0.3 * ref_a.device_ms / 1e3)
                if srv.poll(a) is not None:
                    break
                srv.suspend(a)
                assert _until(srv, "suspended", 1) or srv.poll(a) is not None
                if srv.stats()["suspended"] == 1:
                    # a's budget lets b in while a is held
                    assert _until(srv, "resident", 1)
                    srv.resume(a)
            ra, rb = srv.wait(a), srv.wait(b)
            assert srv.stats()["suspensions"] >= 1
    _same(ra, ref_a)
    _same(rb, ref_b)


def test_suspend_queued_request_and_errors():
    A = W.laplacian_2d(200, shift=0.1)
    with B.Handle.from_csr(A) as h:
        ref = h.oslq(30, 40, seed=9)
        with B.Server(8 << 30, max_slots=1) as srv:
            a = srv.submit(h, B.METHOD_OSLQ, 30, 200, seed=8)
            q = srv.submit(h, B.METHOD_OSLQ, 30, 40, seed=9)
            srv.suspend(q)                       # still queued behind a
            assert srv.stats()["suspended"] == 1
            srv.wait(a)
            time.sleep(0.05)
            assert srv.poll(q) is None           # held: never admitted
            srv.resume(q)
            _same(srv.wait(q), ref)
            with pytest.raises(B.LogdetError) as e:
                srv.suspend(q)                   # finished
            assert e.value.code == B.EINVAL
            with pytest.raises(B.LogdetError) as e:
                srv.resume(a)                    # not suspended
            assert e.value.code == B.EINVAL
            with pytest.raises(B.LogdetError) as e:
                srv.suspend(12345)
            assert e.value.code == B.ENOENT
            # a suspended request can be cancelled
            c = srv.submit(h, B.METHOD_OSLQ, 30, 40, seed=10)
            srv.suspend(c)
            assert _until(srv, "suspended", 1) or srv.poll(c) is not None
            if srv.stats()["suspended"] == 1:
                srv.cancel(c)
                with pytest.raises(B.LogdetError) as e:
                    srv.wait(c)
                assert e.value.code == B.ECANCEL
            assert srv.stats()["suspended"] == 0


def test_server_honours_block_width():
    # the request's block_width reaches the solve (bit-identical to blocking)
    A = W.laplacian_2d(90, 70, shift=0.05)
    with B.Handle.from_csr(A) as h:
        ref = h.oslq(30, 20, seed=3, block_width=10)
        with B.Server(8 << 30, max_slots=2) as srv:
            got = srv.wait(srv.submit(h, B.METHOD_OSLQ, 30, 20, seed=3, block_width=10))
    _same(got, ref)


def test_server_request_log(tmp_path):
    import json
    A = W.laplacian_2d(120, shift=0.1)
    path = tmp_path / "requests.jsonl"
    with B.Handle.from_csr(A) as h:
        with B.Server(8 << 30, max_slots=4) as srv:
            srv.set_log(path)
            ids = [srv.submit(h, B.METHOD_OSLQ, 30, 20, seed=s) for s in range(3)]
            ids.append(srv.submit(h, B.METHOD_OSAIOP, 30, 16, 2, seed=5, precision=B.MIXED_FP32))
            res = [srv.wait(i) for i in ids]
            srv.set_log(None)
    recs = {r["id"]: r for r in map(json.loads, path.read_text().splitlines())}
    assert sorted(recs) == sorted(ids)
    for i, r in zip(ids, res):
        rec = recs[i]
        assert rec["state"] == "done" and rec["rc"] == 0
        assert rec["n"] == A.n and rec["nnz"] == A.nnz
        assert rec["logdet"] == r.logdet and rec["steps_max"] == r.steps_max
        assert rec["latency_ms"] >= rec["queue_ms"] >= 0.0
    assert recs[ids[-1]]["method"] == "osaiop" and recs[ids[-1]]["precision"] == B.MIXED_FP32
