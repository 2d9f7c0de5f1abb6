"""Graph plans (logdet_plan_*): a solve captured once into a CUDA graph and
replayed per seed must give bit-identical results to the blocking entry
points with the same seed and options, and (FP64) agree with the oracle at
the FP64 bar.  Each replay must count its kernels in the launch counter."""
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
    assert a.tr_sub == b.tr_sub and a.tr_res == b.tr_res
    assert np.array_equal(a.per_probe, b.per_probe)
    assert np.array_equal(a.z_norm2, b.z_norm2)
    assert (a.s_eff, a.steps_min, a.steps_max, a.status_bits) == \
        (b.s_eff, b.steps_min, b.steps_max, b.status_bits)


CASES = [
    # (id, matrix maker, method, P, m, k, options)
    ("oslq-2d-fp64", lambda: W.laplacian_2d(64, shift=0.1), 0, 30, 30, 0, {}),
    ("osaiop-3d-k4-fp64", lambda: W.laplacian_3d(20, shift=0.05), 1, 24, 20, 4, {}),
    ("oslq-matern-fp32", lambda: W.matern_2d(40, kappa2=0.05), 0, 30, 25, 0,
     {"precision": B.MIXED_FP32}),
    ("osaiop-fp32-k2", lambda: W.laplacian_2d(50, 31, shift=0.2), 1, 21, 15, 2,
     {"precision": B.MIXED_FP32}),
    ("oslq-plain-gauss", lambda: W.laplacian_2d(33, shift=0.3), 0, 12, 20, 0,
     {"plain": 1, "gaussian": 1}),
    ("osaiop-shift", lambda: W.powerlaw_graph_laplacian(3001, seed=4), 1, 18, 16, 4,
     {"shift": 0.05}),
    ("oslq-autotune", lambda: W.laplacian_3d(24, shift=0.02), 0, 40, 20, 0, {"autotune": 1}),
]


@pytest.mark.parametrize("cid,maker,method,P,m,k,kw", CASES, ids=[c[0] for c in CASES])
def test_plan_replay_bit_identical_to_blocking(cid, maker, method, P, m, k, kw):
    A = maker()
    with B.Handle.from_csr(A) as h:
        blocking = h.oslq if method == 0 else h.osaiop
        with B.Plan(h, method, P, m, k, **kw) as plan:
            nk = plan.kernels()
            assert nk > 0
            for seed in (0, 7, 123456789):
                c0 = B.logdet_launch_count()
                got = plan.run(seed)
                assert B.logdet_launch_count() - c0 == nk
                if method == 0:
                    want = blocking(P, m, seed=seed, iop_window=k, **kw)
                else:
                    want = blocking(P, m, iop_window=k, seed=seed, **kw)
                _same(got, want)


def test_plan_matches_oracle_fp64():
    A = W.laplacian_2d(64, shift=0.1)
    with B.Handle.from_csr(A) as h, B.Plan(h, 0, 30, 30) as plan:
        for seed in (3, 4):
            got = plan.run(seed)
            want = O.oslq(A.to_scipy(), 30, 30, seed=seed)
            assert abs(got.logdet - want.logdet) <= 1e-10 * abs(want.logdet)
            assert np.allclose(got.per_probe, want.per_probe, rtol=0, atol=1e-9)


def test_plan_on_user_stream_and_interleaved_plans():
    A = W.laplacian_2d(48, shift=0.1)
    s = torch.cuda.Stream()
    with B.Handle.from_csr(A) as h:
        with B.Plan(h, 0, 30, 20, stream=s) as p1, B.Plan(h, 1, 30, 20, 4, stream=s) as p2:
            r1 = [p1.run(i) for i in range(3)]
            r2 = [p2.run(i) for i in range(3)]
            r1b = [p1.run(i) for i in range(3)]
        for i in range(3):
            _same(r1[i], r1b[i])
            _same(r1[i], h.oslq(30, 20, seed=i))
            _same(r2[i], h.osaiop(30, 20, iop_window=4, seed=i))


def test_plan_invalid_arguments():
    A = W.laplacian_2d(16, shift=0.1)
    with B.Handle.from_csr(A) as h:
        with pytest.raises(B.LogdetError):
            B.Plan(h, 0, 2, 10)          # num_probes < 3
        with pytest.raises(B.LogdetError):
            B.Plan(h, 2, 30, 10)         # unknown method
        with pytest.raises(B.LogdetError):
            B.Plan(h, 0, 30, A.n + 1)    # krylov_steps > n
