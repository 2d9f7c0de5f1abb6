"""Double-float Krylov vectors (LOGDET_MIXED_F32X2) through the C-ABI.

The mode keeps the matrix values in FP32 (the scaled values Q_ij / c rounded
once, as the mixed FP32 path) and stores every Krylov vector as a pair of
floats hi + lo, computed on in double-float arithmetic (error-free TwoSum and
FMA TwoProduct on the FP32 pipe, about 2^-44 relative per operation).  What
it computes is therefore the estimator of the FP32-rounded matrix at close to
FP64 precision, and the tests pin exactly that:

  - against the oracle run on the rounded matrix (entries fl32(Q_ij / c) c,
    the same spectral interval passed to both sides so that c agrees) the
    log-determinant agrees to 1e-8 relative: 2^-44 per operation, amplified
    by the recurrence's sensitivity to rounding (about 7e3 on the worst
    workloads for FP32 vectors) stays below 1e-9;
  - against the oracle on the exact matrix it is within the mixed budget
    1e-4 (the FP32 value rounding perturbs each entry by at most 2^-24 of
    itself);
  - shift groups, the server, plans and autotuned or forced layouts take
    the mode like the other precisions; gridded operators refuse it.
"""
import math

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

RTOL_ROUNDED = 1e-8
RTOL_MIXED = 1e-4
DF = B.MIXED_F32X2


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def rounded(Q, c):
    """The matrix the FP32 values stand for: fl32(Q_ij / c) * c."""
    R = Q.copy().tocsr()
    R.data = (R.data / c).astype(np.float32).astype(np.float64) * c
    return R


def scale_of(method, lam):
    return lam[1] if method == "oslq" else math.sqrt(lam[0] * lam[1])


def _pair(A, method, P, m, k, seed):
    """(GPU double-float result, oracle on the rounded matrix, oracle on A)."""
    Q = A.to_scipy()
    lam = O.spectral_interval(Q)
    Qr = rounded(Q, scale_of(method, lam))
    with B.Handle.from_csr(A) as h:
        if method == "oslq":
            res = h.oslq(P, m, seed=seed, lam=lam, precision=DF)
            er = O.oslq(Qr, P, m, seed=seed, lam=lam)
            ex = O.oslq(Q, P, m, seed=seed, lam=lam)
        else:
            res = h.osaiop(P, m, iop_window=k, seed=seed, lam=lam, precision=DF)
            er = O.osaiop(Qr, P, m, k=k, seed=seed, lam=lam)
            ex = O.osaiop(Q, P, m, k=k, seed=seed, lam=lam)
    return res, er, ex


def test_oslq_64x64_laplacian_parity():
    res, er, ex = _pair(W.laplacian_2d(64, shift=0.1), "oslq", 30, 30, 0, 0)
    assert (res.s, res.r, res.s_eff) == (er.s, er.r, er.s_eff)
    assert res.steps_max == 30
    assert rel(res.logdet, er.logdet) <= RTOL_ROUNDED
    assert rel(res.tr_res, er.tr_res) <= 1e-7
    assert rel(res.logdet, ex.logdet) <= RTOL_MIXED


@pytest.mark.parametrize("k", [2, 4, 8])
def test_osaiop_parity(k):
    res, er, ex = _pair(W.laplacian_2d(40, 37, shift=0.05), "osaiop", 30, 25, k, 3)
    assert rel(res.logdet, er.logdet) <= RTOL_ROUNDED
    assert rel(res.logdet, ex.logdet) <= RTOL_MIXED


@pytest.mark.parametrize("method,k", [("oslq", 0), ("osaiop", 3)])
def test_ragged_sizes_and_odd_probe_count(method, k):
    # n = 990 (several tiles and a ragged tail), 31 probes: s = 10, r = 11,
    # block width 21 padded to 22 (two double-float entries per vector)
    res, er, _ = _pair(W.laplacian_3d(11, 9, 10, shift=0.02), method, 31, 17, k, 9)
    assert (res.s, res.r) == (10, 11)
    assert rel(res.logdet, er.logdet) <= RTOL_ROUNDED


def test_ill_conditioned_powerlaw_graph():
    # Graph Laplacian of a power-law graph (hub rows split into work items)
    # with the smallest shift of the batched workload, 1e-3: the case whose
    # FP32-vector error exceeds the 1e-4 budget at full size.
    A = W.powerlaw_graph_laplacian(30011, exponent=2.3, mean_degree=8.0,
                                   seed=4).with_diagonal_shift(1e-3)
    res, er, ex = _pair(A, "osaiop", 24, 40, 4, 5)
    assert rel(res.logdet, er.logdet) <= RTOL_ROUNDED
    assert rel(res.logdet, ex.logdet) <= RTOL_MIXED
    with B.Handle.from_csr(A) as h:
        r32 = h.osaiop(24, 40, iop_window=4, seed=5, lam=O.spectral_interval(A.to_scipy()),
                       precision=B.MIXED_FP32)
    # the double-float vectors are closer to the rounded matrix's estimate
    # than the FP32 vectors are
    assert rel(res.logdet, er.logdet) < rel(r32.logdet, er.logdet)


def test_identity_and_tiny_matrix():
    with B.Handle.from_csr(W.scaled_identity(300, 2.5)) as h:
        r = h.oslq(9, 10, precision=DF)   # 2.5 / c is exact in FP32 for c = 2.5
    assert r.steps_max == 1 and r.status_bits & B.ST_BREAKDOWN
    assert r.logdet == pytest.approx(300 * math.log(2.5), rel=1e-13)
    A = W.laplacian_2d(3, shift=1.0)      # n = 9, s = 9 >= n: residual vanishes
    res, er, _ = _pair(A, "oslq", 29, 7, 0, 1)
    assert res.s_eff == er.s_eff
    assert rel(res.logdet, er.logdet) <= RTOL_ROUNDED


def test_autotuned_and_forced_layouts():
    A = W.laplacian_2d(70, 61, shift=0.05)
    with B.Handle.from_csr(A) as h:
        base = h.osaiop(30, 20, iop_window=4, seed=2, precision=DF)
        tuned = h.osaiop(30, 20, iop_window=4, seed=2, precision=DF, autotune=1)
        sliced = h.osaiop(30, 20, iop_window=4, seed=2, precision=DF, block_width=2)
        with pytest.raises(B.LogdetError):   # not a multiple of the 2-entry vector
            h.osaiop(30, 20, iop_window=4, seed=2, precision=DF, block_width=3)
    # other tilings change the order of the dot partials only
    assert rel(tuned.logdet, base.logdet) <= 1e-11
    assert rel(sliced.logdet, base.logdet) <= 1e-11


@pytest.mark.parametrize("method,k", [(0, 0), (1, 3)])
def test_shift_group_members(method, k):
    A = W.laplacian_2d(45, 37, shift=0.0)
    shifts = [0.05, 0.4, 1.0, 3.0]
    P, m, seed0 = 30, 25, 11
    Q = A.to_scipy()
    I = sp.identity(A.n, format="csr")
    with B.Handle.from_csr(A) as h:
        if method == 0:
            grp = h.oslq_shifts(shifts, P, m, seed0=seed0, precision=DF)
            own = [h.oslq(P, m, seed=seed0 + t, shift=s, precision=DF) for t, s in enumerate(shifts)]
        else:
            grp = h.osaiop_shifts(shifts, P, m, iop_window=k, seed0=seed0, precision=DF)
            own = [h.osaiop(P, m, iop_window=k, seed=seed0 + t, shift=s, precision=DF)
                   for t, s in enumerate(shifts)]
    for t, s in enumerate(shifts):
        # members round member 0's scaled values: their FP32 matrices differ
        # from their own solves' by value rounding only
        assert rel(grp[t].logdet, own[t].logdet) <= 1e-6, t
        Qs = (Q + s * I).tocsr()
        est = (O.oslq(Qs, P, m, seed=seed0 + t) if method == 0
               else O.osaiop(Qs, P, m, k=k, seed=seed0 + t))
        assert rel(grp[t].logdet, est.logdet) <= RTOL_MIXED, t


def test_plan_replays_the_blocking_solve():
    A = W.laplacian_3d(16, 15, 14, shift=0.05)
    with B.Handle.from_csr(A) as h:
        want = [h.osaiop(21, 12, iop_window=2, seed=s, precision=DF) for s in (4, 5)]
        with B.Plan(h, B.METHOD_OSAIOP, 21, 12, 2, precision=DF) as p:
            got = [p.run(s) for s in (4, 5)]
    for w, g in zip(want, got):
        assert g.logdet == w.logdet


@pytest.mark.parametrize("method,k", [("oslq", 0), ("osaiop", 3)])
def test_plain_slq_gaussian_probes_and_tol_mode(method, k):
    # the options that change the path (no sketch; Gaussian probes; the
    # tol = 1e-6 early stop) against the oracle on the rounded matrix
    A = W.laplacian_2d(40, 35, shift=0.2)
    Q = A.to_scipy()
    lam = O.spectral_interval(Q)
    Qr = rounded(Q, scale_of(method, lam))
    kw = {} if method == "oslq" else {"iop_window": k}
    okw = {} if method == "oslq" else {"k": k}
    f = O.oslq if method == "oslq" else O.osaiop
    with B.Handle.from_csr(A) as h:
        g = h.oslq if method == "oslq" else h.osaiop
        rp = g(20, 25, seed=2, lam=lam, precision=DF, plain=1, **kw)
        rg = g(30, 20, seed=5, lam=lam, precision=DF, gaussian=1, **kw)
        rt = g(21, 40, seed=3, lam=lam, precision=DF, tol=1e-6, **kw)
    ep = f(Qr, 20, 25, seed=2, lam=lam, hutchpp=False, **okw)
    eg = f(Qr, 30, 20, seed=5, lam=lam, gaussian=True, **okw)
    et = f(Qr, 21, 40, seed=3, lam=lam, tol=1e-6, **okw)
    assert (rp.s, rp.r) == (0, 20)
    assert rel(rp.logdet, ep.logdet) <= RTOL_ROUNDED
    assert rel(rg.logdet, eg.logdet) <= RTOL_ROUNDED
    assert rel(rt.logdet, et.logdet) <= RTOL_ROUNDED
    assert rt.steps_max <= 40
