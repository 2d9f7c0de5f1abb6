"""The persistent Krylov run (opt-in, LOGDET_KRYLOV_PERSISTENT=1): for small
blocks every step of a Krylov phase (pass 1, the coefficients, pass 2, the
norms) runs in one cooperative launch, with bounded grid barriers.  Its
results must be bit-identical to the step-by-step path (the default), match
the FP64 oracle, replay bit-identically from a graph plan, and a barrier wait
that runs out must fail the solve with LOGDET_ETIMEOUT and leave the context
usable."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_07004_gb300 import binding as B  # noqa: E402


def _same(a, b):
    assert a.logdet == b.logdet
    assert np.array_equal(a.per_probe, b.per_probe)
    assert np.array_equal(a.z_norm2, b.z_norm2)
    assert (a.steps_min, a.steps_max, a.status_bits) == (b.steps_min, b.steps_max, b.status_bits)


def _runs(h, method, k, **kw):
    if method == "oslq":
        return h.oslq(30, 30, seed=3, **kw)
    return h.osaiop(30, 30, iop_window=k, seed=3, **kw)


CASES = [("oslq", 0, B.FP64), ("osaiop", 1, B.FP64), ("osaiop", 2, B.FP64), ("osaiop", 4, B.FP64),
         ("osaiop", 8, B.FP64), ("oslq", 0, B.MIXED_FP32), ("osaiop", 4, B.MIXED_FP32)]


@pytest.mark.parametrize("method,k,prec", CASES)
def test_persistent_run_equals_step_path(method, k, prec, monkeypatch):
    # 2D Laplacian 50 x 47 (n = 2350, below the size that takes the line
    # sweep): every Krylov phase qualifies for the persistent run.
    A = W.laplacian_2d(50, 47, shift=0.05)
    with B.Handle.from_csr(A) as h:
        monkeypatch.setenv("LOGDET_KRYLOV_PERSISTENT", "1")
        B.logdet_profile_reset()
        B.logdet_profile_enable(True)
        fast = _runs(h, method, k, precision=prec)
        B.logdet_profile_enable(False)
        prof = B.profile_snapshot()
        monkeypatch.setenv("LOGDET_KRYLOV_PERSISTENT", "0")
        steps = _runs(h, method, k, precision=prec)
    _same(fast, steps)
    # one launch per Krylov phase, no step kernels
    assert prof["krylov_run"]["launches"] == (1 if method == "oslq" else 2)
    assert prof["spmm"]["launches"] <= 1 and prof["update"]["launches"] == 0


def test_persistent_run_matches_oracle_and_variants(monkeypatch):
    # The 64^2 Laplacian + 0.1 I workload (OSLQ m = 30, 30 probes) and the
    # other solve variants: plain SLQ, Gaussian probes, a diagonal shift,
    # an odd probe count (ragged block), each against the step path.
    A = W.laplacian_2d(64, shift=0.1)
    Q = A.to_scipy()
    est = O.oslq(Q, 30, 30, seed=0)
    monkeypatch.setenv("LOGDET_KRYLOV_PERSISTENT", "1")
    with B.Handle.from_csr(A) as h:
        res = h.oslq(30, 30, seed=0)
        assert abs(res.logdet - est.logdet) / abs(est.logdet) <= 1e-10
        variants = [dict(plain=1), dict(gaussian=1), dict(shift=0.37)]
        got = [h.oslq(31, 25, seed=5, **v) for v in variants]
        got += [h.osaiop(31, 25, iop_window=3, seed=5, **v) for v in variants]
        monkeypatch.setenv("LOGDET_KRYLOV_PERSISTENT", "0")
        want = [h.oslq(31, 25, seed=5, **v) for v in variants]
        want += [h.osaiop(31, 25, iop_window=3, seed=5, **v) for v in variants]
    for a, b in zip(got, want):
        _same(a, b)


def test_persistent_run_breakdown_and_single_step(monkeypatch):
    # Breakdown at step 1 (Q = c I) and m = 1 (no pass 2 at all).
    monkeypatch.setenv("LOGDET_KRYLOV_PERSISTENT", "1")
    A = W.scaled_identity(3000, 2.5)
    with B.Handle.from_csr(A) as h:
        r = h.oslq(9, 10)
        assert r.steps_max == 1 and r.status_bits & B.ST_BREAKDOWN
        assert r.logdet == pytest.approx(3000 * np.log(2.5), rel=1e-13)
    A = W.laplacian_2d(30, shift=0.2)
    est = O.oslq(A.to_scipy(), 12, 1, seed=2)
    with B.Handle.from_csr(A) as h:
        r = h.oslq(12, 1, seed=2)
    assert abs(r.logdet - est.logdet) / abs(est.logdet) <= 1e-10


def test_plan_replays_persistent_run_bit_identically(monkeypatch):
    # plans captured with the persistent run, against blocking step-path solves
    A = W.laplacian_2d(64, shift=0.1)
    with B.Handle.from_csr(A) as h:
        monkeypatch.setenv("LOGDET_KRYLOV_PERSISTENT", "1")
        p1 = B.Plan(h, B.METHOD_OSLQ, 30, 30)
        p2 = B.Plan(h, B.METHOD_OSAIOP, 30, 20, iop_window=4)
        monkeypatch.delenv("LOGDET_KRYLOV_PERSISTENT")
        with p1, p2:
            assert p1.kernels() < 40
            for seed in (0, 11):
                _same(p1.run(seed), h.oslq(30, 30, seed=seed))
            _same(p2.run(4), h.osaiop(30, 20, iop_window=4, seed=4))


def test_barrier_wait_timeout_reports_and_recovers(monkeypatch):
    # LOGDET_TEST_KRUN_STALL=1 makes every grid barrier wait for one CTA more
    # than the grid has, with a 20 ms bound: every wait runs out, the CTAs
    # flag the run and return.  The solve fails with LOGDET_ETIMEOUT; the
    # next solve on the same handle is exact.
    A = W.laplacian_2d(40, shift=0.05)
    monkeypatch.setenv("LOGDET_KRYLOV_PERSISTENT", "1")
    with B.Handle.from_csr(A) as h:
        want = h.oslq(30, 12, seed=1)
        monkeypatch.setenv("LOGDET_TEST_KRUN_STALL", "1")
        with pytest.raises(B.LogdetError) as e:
            h.oslq(30, 12, seed=1)
        assert e.value.code == B.ETIMEOUT
        monkeypatch.delenv("LOGDET_TEST_KRUN_STALL")
        _same(h.oslq(30, 12, seed=1), want)
