"""Full-size workloads, in the launch configuration the benchmark times.

The oracle cannot run whole solves at these sizes within a test, so it
computes sampled outputs one by one: the Hutch++ split (every |z_j|^2) and the
quadrature forms of sampled probes, compared with the CUDA path's per-probe
outputs.  The mixed path is compared with the FP64 CUDA path (same seed).
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_07004_gb300 import binding as B  # noqa: E402


@pytest.fixture(scope="module")
def lap3d():
    A = W.laplacian_3d(128, shift=0.01)
    with B.Handle.from_csr(A) as h:
        yield A, h


def _oracle_split(Q, J_or_L_sketch, s, r, seed):
    n = Q.shape[0]
    S = O.rademacher_block(seed, 0, n, s)
    G = O.rademacher_block(seed, 1, n, r)
    Y = J_or_L_sketch(S)
    A = O.orth(Y)
    Z = G - A @ (A.T @ G)
    return A, Z


def test_oslq_128cubed_sampled_probes(lap3d):
    A, h = lap3d
    Q = A.to_scipy()
    res = h.oslq(60, 50, seed=1000)
    lo, hi = O.spectral_interval(Q)
    J = Q / hi
    Aq, Z = _oracle_split(Q, lambda S: J @ S, 20, 20, 1000)
    zn2 = np.einsum("ij,ij->j", Z, Z)
    np.testing.assert_allclose(res.z_norm2, zn2, rtol=1e-11)
    for i in (0, 13):                      # two range probes
        al, be = O.lanczos(J, Aq[:, i], 50)
        want = O.gauss_quadrature_log(al, be).value
        assert abs(res.per_probe[i] - want) <= 1e-9 * max(1.0, abs(want)), i
    for j in (0, 19):                      # two residual probes
        al, be = O.lanczos(J, Z[:, j], 50)
        want = O.gauss_quadrature_log(al, be).value
        assert abs(res.per_probe[20 + j] - want) <= 1e-9 * max(1.0, abs(want)), j
    assert res.steps_min == res.steps_max == 50
    # the estimate itself is within the estimator's own error of the closed form
    exact = W.closed_form_logdet_laplacian_3d(128, shift=0.01)
    assert abs(res.logdet - exact) / exact < 5e-3


@pytest.fixture(scope="module")
def oracle_pool():
    from oracle_pool import make_pool
    pool = make_pool()
    yield pool
    pool.close()
    pool.join()


@pytest.mark.parametrize("k", [2, 4, 8])
def test_osaiop_128cubed_sampled_probes(lap3d, oracle_pool, k):
    # The benchmark's OSA-IOP solves (60 probes, m = 50, windows 2, 4, 8):
    # the wide-window kernel instances run here with the deep tiles of the
    # full-size launch.
    from oracle_pool import iop_actions
    A, h = lap3d
    res = h.osaiop(60, 50, iop_window=k, seed=1000)
    spec = ("laplacian_3d", (128, 0.01))
    # The oracle builds the whole Hutch++ split itself (20 Algorithm-1 actions
    # for Y = L S), then checks every |z_j|^2 and the forms of sampled probes.
    S = O.rademacher_block(1000, 0, A.n, 20)
    Y = np.stack(iop_actions(oracle_pool, spec, S, 50, k), axis=1)
    Aq = O.orth(Y)
    G = O.rademacher_block(1000, 1, A.n, 20)
    Z = G - Aq @ (Aq.T @ G)
    np.testing.assert_allclose(res.z_norm2, np.einsum("ij,ij->j", Z, Z), rtol=1e-9)
    probes = np.stack([Z[:, 0], Z[:, 7], Z[:, 19], Aq[:, 3], Aq[:, 16]], axis=1)
    LZ = iop_actions(oracle_pool, spec, probes, 50, k)
    for col, j in enumerate((0, 7, 19)):
        want = float(Z[:, j] @ LZ[col]) / float(Z[:, j] @ Z[:, j])
        assert abs(res.per_probe[20 + j] - want) <= 1e-9 * max(1.0, abs(want)), (k, j)
    for col, i in ((3, 3), (4, 16)):
        qf = float(Aq[:, i] @ LZ[col])
        assert abs(res.per_probe[i] - qf) <= 1e-9 * max(1.0, abs(qf)), (k, i)
    assert res.steps_min == res.steps_max == 50
    exact = W.closed_form_logdet_laplacian_3d(128, shift=0.01)
    assert abs(res.logdet - exact) / exact < 5e-3


def test_matern_mixed_within_1e4_of_fp64():
    A = W.matern_2d(1024, 0.05, dtype=np.float32)
    with B.Handle.from_csr(A) as h:
        r32 = h.oslq(120, 80, seed=7, precision=B.MIXED_FP32)
        r64 = h.oslq(120, 80, seed=7, precision=B.FP64)
    assert abs(r32.logdet - r64.logdet) / abs(r64.logdet) <= 1e-4
    exact = W.closed_form_logdet_matern_2d(1024, 0.05)
    assert abs(r64.logdet - exact) / exact < 1e-2
