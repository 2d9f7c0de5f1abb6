"""Shift groups (logdet_oslq_shifts / logdet_osaiop_shifts) through the C-ABI.

Member t of a group is by definition the solve of log det(Q + shifts[t] I)
with seed seed0 + t; the group only changes how its Krylov phases are run
(one run over all members' columns, each column with its own diagonal shift
and scale).  So:
  - a group of one is bit-identical to the ordinary solve (the column scale
    is exactly 1 and every sum keeps its order);
  - in FP64 each member is within 1e-12 of its ordinary solve (one rounding
    more per SpMM: (Q/c_0 + shift/c_0) x c_0/c_t) and within 1e-10 of the
    oracle on Q + shift I;
  - mixed FP32 members are within 1e-5 of their ordinary mixed solve on
    well-conditioned operators, and within the 1e-4 mixed band of FP64;
  - malformed groups are refused with EINVAL.
"""
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


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def _single(h, method, P, m, k, seed, shift, **kw):
    if method == 0:
        return h.oslq(P, m, seed=seed, shift=shift, **kw)
    return h.osaiop(P, m, iop_window=k, seed=seed, shift=shift, **kw)


def _group(h, method, shifts, P, m, k, seed0, **kw):
    if method == 0:
        return h.oslq_shifts(shifts, P, m, seed0=seed0, **kw)
    return h.osaiop_shifts(shifts, P, m, iop_window=k, seed0=seed0, **kw)


@pytest.mark.parametrize("method,k", [(0, 0), (1, 2), (1, 4)])
@pytest.mark.parametrize("precision", [B.FP64, B.MIXED_FP32, B.MIXED_BF16VEC, B.MIXED_F32X2])
@pytest.mark.parametrize("plain", [0, 1])
def test_group_of_one_is_the_ordinary_solve(method, k, precision, plain):
    A = W.laplacian_2d(61, 47, shift=0.0)
    with B.Handle.from_csr(A) as h:
        g = _group(h, method, [0.35], 31, 24, k, 5, precision=precision, plain=plain)
        o = _single(h, method, 31, 24, k, 5, 0.35, precision=precision, plain=plain)
    assert len(g) == 1
    assert g[0].logdet == o.logdet
    assert (g[0].tr_sub, g[0].tr_res, g[0].s_eff) == (o.tr_sub, o.tr_res, o.s_eff)
    assert (g[0].steps_min, g[0].steps_max, g[0].status_bits) == (o.steps_min, o.steps_max,
                                                                   o.status_bits)


@pytest.mark.parametrize("method,k", [(0, 0), (1, 2), (1, 3)])
@pytest.mark.parametrize("P", [30, 31])  # 31: FP64 block 21 columns wide, padded to 22
def test_fp64_members_equal_their_own_solves_and_the_oracle(method, k, P):
    A = W.laplacian_2d(45, 37, shift=0.0)
    shifts = [0.05, 0.4, 1.0, 3.0]
    m, seed0 = 25, 11
    with B.Handle.from_csr(A) as h:
        grp = _group(h, method, shifts, P, m, k, seed0)
        own = [_single(h, method, P, m, k, seed0 + t, sh) for t, sh in enumerate(shifts)]
    Q = A.to_scipy()
    I = sp.identity(A.n, format="csr")
    for t, sh in enumerate(shifts):
        assert rel(grp[t].logdet, own[t].logdet) <= 1e-12, t
        assert (grp[t].s_eff, grp[t].steps_max) == (own[t].s_eff, own[t].steps_max)
        Qs = (Q + sh * I).tocsr()
        est = (O.oslq(Qs, P, m, seed=seed0 + t) if method == 0
               else O.osaiop(Qs, P, m, k=k, seed=seed0 + t))
        assert rel(grp[t].logdet, est.logdet) <= 1e-10, t
        # the exact value for orientation: a 1.7k-row Laplacian has it cheaply
        exact = np.linalg.slogdet(Qs.toarray())[1]
        assert rel(grp[t].logdet, exact) <= 5e-2


@pytest.mark.parametrize("method,k", [(0, 0), (1, 4)])
def test_mixed_members_within_1e5_of_their_own_and_1e4_of_fp64(method, k):
    # m = 40 steps on a 2D Laplacian (n = 16384, padded FP32 sketch block:
    # s = 21 of 24 columns) and 6 shifts: 6 x 44 = 264 block columns
    A = W.laplacian_2d(128, shift=0.0)
    shifts = [0.02, 0.05, 0.1, 0.3, 1.0, 2.5]
    P, m, seed0 = 64, 40, 3
    with B.Handle.from_csr(A) as h:
        grp = _group(h, method, shifts, P, m, k, seed0, precision=B.MIXED_FP32)
        own = [_single(h, method, P, m, k, seed0 + t, sh, precision=B.MIXED_FP32)
               for t, sh in enumerate(shifts)]
        g64 = _group(h, method, shifts, P, m, k, seed0)
    for t in range(len(shifts)):
        assert rel(grp[t].logdet, own[t].logdet) <= 1e-5, t
        assert rel(grp[t].logdet, g64[t].logdet) <= 1e-4, t
    assert np.all(np.diff([r.logdet for r in g64]) > 0)


def test_irregular_graph_group_matches_own_solves():
    # power-law graph Laplacian: the SpMM runs on work items (irregular rows)
    A = W.powerlaw_graph_laplacian(30011, exponent=2.3, mean_degree=8.0, seed=4)
    shifts = [1e-2, 3e-2, 1e-1]
    P, m, k = 24, 30, 4
    with B.Handle.from_csr(A) as h:
        g64 = h.osaiop_shifts(shifts, P, m, iop_window=k, seed0=0)
        o64 = [h.osaiop(P, m, iop_window=k, seed=t, shift=sh) for t, sh in enumerate(shifts)]
        g32 = h.osaiop_shifts(shifts, P, m, iop_window=k, seed0=0, precision=B.MIXED_FP32)
    for t in range(len(shifts)):
        assert rel(g64[t].logdet, o64[t].logdet) <= 1e-10, t
        assert rel(g32[t].logdet, g64[t].logdet) <= 1e-3, t


def test_group_reuses_nothing_between_calls():
    A = W.laplacian_3d(14, shift=0.0)
    with B.Handle.from_csr(A) as h:
        a = h.oslq_shifts([0.1, 0.2], 12, 15, seed0=7)
        b = h.oslq_shifts([0.1, 0.2], 12, 15, seed0=7)
        c = h.oslq_shifts([0.2], 12, 15, seed0=8)
    assert [r.logdet for r in a] == [r.logdet for r in b]
    assert c[0].logdet == pytest.approx(a[1].logdet, rel=1e-12)


def test_malformed_groups_refused():
    A = W.laplacian_2d(20, shift=0.0)
    with B.Handle.from_csr(A) as h:
        with pytest.raises(B.LogdetError) as e:
            h.oslq_shifts([], 12, 10)
        assert e.value.code == B.EINVAL
        with pytest.raises(B.LogdetError) as e:
            h.oslq_shifts([0.1, -1.0], 12, 10)
        assert e.value.code == B.EINVAL
    with B.Handle.grid(24, 24, np.array([[4.5, -1.0], [-1.0, 0.0]])) as hg:
        with pytest.raises(B.LogdetError) as e:
            hg.oslq_shifts([0.1, 0.2], 12, 10)
        assert e.value.code == B.EINVAL


@pytest.mark.parametrize("nshift", [23, 24, 47])
def test_wide_groups_split_into_runs(nshift):
    # 44 FP64 block columns per member and at most 1024 per run: 23 shifts
    # run together (1012 columns, the widest tile geometry), 24 as two runs
    # of 12, 47 as 16 + 16 + 15
    A = W.laplacian_2d(20, shift=0.0)
    shifts = np.linspace(0.1, 1.0, nshift)
    with B.Handle.from_csr(A) as h:
        r = h.osaiop_shifts(shifts, 64, 6, iop_window=2, seed0=5)
        own = [h.osaiop(64, 6, iop_window=2, seed=5 + t, shift=float(sh))
               for t, sh in enumerate(shifts)]
    assert len(r) == nshift
    for t in range(nshift):
        assert rel(r[t].logdet, own[t].logdet) <= 1e-12, t


@pytest.mark.parametrize("method,k", [(0, 0), (1, 2)])
def test_group_breakdown_and_tiny_matrices(method, k):
    # identity: every probe breaks down after one step, in every member
    A = W.scaled_identity(300, 2.5)
    shifts = [0.0, 0.5, 4.0]
    with B.Handle.from_csr(A) as h:
        g = _group(h, method, shifts, 9, 10, k, 0)
    for t, sh in enumerate(shifts):
        assert g[t].steps_max == 1 and g[t].status_bits & B.ST_BREAKDOWN
        assert g[t].logdet == pytest.approx(300 * np.log(2.5 + sh), rel=1e-13)
    # 5 distinct diagonal values: every run breaks down at the distinct count
    d = np.repeat([0.5, 1.0, 2.0, 3.5, 7.0], 40)
    A = W.diagonal_matrix(d)
    with B.Handle.from_csr(A) as h:
        g = _group(h, method, shifts, 12, 8, k, 2)
        own = [_single(h, method, 12, 8, k, 2 + t, sh) for t, sh in enumerate(shifts)]
    for t, sh in enumerate(shifts):
        assert rel(g[t].logdet, own[t].logdet) <= 1e-12
        assert (g[t].steps_max, g[t].status_bits) == (own[t].steps_max, own[t].status_bits)
    # n = 9 with 29 probes: the sketch has rank n, the residual vanishes
    A = W.laplacian_2d(3, shift=1.0)
    with B.Handle.from_csr(A) as h:
        g = _group(h, method, shifts, 29, 7, k, 1)
        own = [_single(h, method, 29, 7, k, 1 + t, sh) for t, sh in enumerate(shifts)]
    for t in range(len(shifts)):
        assert g[t].s_eff == own[t].s_eff
        assert rel(g[t].logdet, own[t].logdet) <= 1e-12


@pytest.mark.parametrize("method,k,precision", [(0, 0, B.FP64), (1, 4, B.MIXED_FP32)])
def test_server_shift_groups_equal_the_blocking_group(method, k, precision):
    # through the server, alongside ordinary requests: each member equals the
    # blocking group call bit for bit, and the ordinary requests their
    # blocking solves
    A = W.laplacian_2d(70, 60, shift=0.0)
    shifts = list(np.linspace(0.05, 1.0, 5))
    with B.Handle.from_csr(A) as h:
        ref = _group(h, method, shifts, 30, 20, k, 4, precision=precision)
        plain_ref = _single(h, method, 30, 20, k, 9, 0.2, precision=precision)
        with B.Server(16 << 30, max_slots=8) as srv:
            other = srv.submit(h, method, 30, 20, k, seed=9, precision=precision, shift=0.2)
            ids = srv.submit_shifts(h, method, shifts, 30, 20, k, seed0=4, precision=precision)
            got = [srv.wait(i) for i in ids]
            plain = srv.wait(other)
            assert srv.stats()["completed"] == len(shifts) + 1
    for a, b in zip(got, ref):
        assert a.logdet == b.logdet
        assert (a.tr_sub, a.tr_res, a.steps_max, a.status_bits) == \
            (b.tr_sub, b.tr_res, b.steps_max, b.status_bits)
    assert plain.logdet == plain_ref.logdet


def test_server_shift_group_runs_cancel_and_suspend():
    A = W.laplacian_2d(20, shift=0.0)
    shifts = np.linspace(0.1, 1.0, 24)          # two runs of 12 (FP64, 44 columns each)
    with B.Handle.from_csr(A) as h:
        ref = h.osaiop_shifts(shifts, 64, 6, iop_window=2, seed0=5)
        with B.Server(16 << 30, max_slots=4) as srv:
            ids = srv.submit_shifts(h, B.METHOD_OSAIOP, shifts, 64, 6, 2, seed0=5)
            got = [srv.wait(i) for i in ids]
            with pytest.raises(B.LogdetError) as e:
                srv.suspend(ids[0])              # finished member
            assert e.value.code == B.EINVAL
            # cancelling one member cancels its run (and nothing else)
            big = W.laplacian_3d(64, shift=0.0)
            with B.Handle.from_csr(big) as hb:
                ids2 = srv.submit_shifts(hb, B.METHOD_OSLQ, [0.1, 0.2, 0.3], 30, 200, seed0=1)
                with pytest.raises(B.LogdetError) as e:
                    srv.suspend(ids2[1])
                assert e.value.code == B.EINVAL
                srv.cancel(ids2[1])
                for i in ids2:
                    with pytest.raises(B.LogdetError) as e:
                        srv.wait(i)
                    assert e.value.code == B.ECANCEL
    assert [r.logdet for r in got] == [r.logdet for r in ref]
