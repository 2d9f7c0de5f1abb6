"""The allocation-free Hessenberg-log entry point against the allocating one.

logdet_hessenberg_log_e1_noalloc serves callers that cannot allocate device
memory while they run (fixed device budgets, external allocators that own all
device memory); it computes on a static scratch array inside the library.
Two calls in a row (the scratch keeps the previous call's contents) must each
match logdet_hessenberg_log_e1 on the same inputs within the 1e-11 tolerance
the Hessenberg-log parity test uses, on both the shared-memory (m <= 80) and
the static-scratch (m >= 81) paths; on the static-scratch path the result is
also checked against SciPy's logm.  The size limit is checked on both sides
of the m = 80 / 81 boundary.  This file sorts last so a run that stops at the
first failure has run every other test first.
"""
import scipy.linalg as sla
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


def _hessenbergs(m, nprobe, k, seed):
    Q = W.laplacian_3d(12, shift=0.02).to_scipy()
    lo, hi = O.spectral_interval(Q)
    Qt = Q / math.sqrt(lo * hi)
    ldh = m + 1
    Hs = np.zeros((nprobe, m, ldh))
    ms = np.zeros(nprobe, dtype=np.int32)
    for p in range(nprobe):
        v = O.rademacher_block(seed + p, 0, Q.shape[0], 1)[:, 0]
        run = O.arnoldi_iop(Qt, v, m - (p % 3), k=k)
        ms[p] = run.m_eff
        Hs[p, :run.m_eff, :run.m_eff] = run.H.T
    return Hs, ms, ldh


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("m,nprobe", [(40, 24), (96, 8), (80, 41), (81, 39)])
def test_noalloc_matches_allocating_entry_point_twice(m, nprobe):
    for call, (k, seed) in enumerate(((2, 10), (4, 50))):
        Hs, ms, ldh = _hessenbergs(m, nprobe, k, seed)
        Hd, md = _dev(Hs.ravel()), _dev(ms, torch.int32)
        c_ref = torch.zeros(nprobe * m, dtype=torch.float64, device="cuda")
        c_new = torch.full((nprobe * m,), float("nan"), dtype=torch.float64, device="cuda")
        st_ref = B.logdet_hessenberg_log_e1(Hd, ldh, md, m, nprobe, c_ref)
        st_new = B.logdet_hessenberg_log_e1_noalloc(Hd, ldh, md, m, nprobe, c_new)
        ref = c_ref.view(nprobe, m).cpu().numpy()
        new = c_new.view(nprobe, m).cpu().numpy()
        assert st_new == st_ref == 0, call
        scale = max(1.0, float(np.max(np.abs(ref))))
        assert np.max(np.abs(new - ref)) <= 1e-11 * scale, call
        if m >= 81:                       # the static-scratch path, against SciPy
            for p in (0, nprobe - 1):
                mp = int(ms[p])
                want = sla.logm(Hs[p, :mp, :mp].T).real[:, 0]
                sc = max(1.0, float(np.max(np.abs(want))))
                assert np.max(np.abs(new[p, :mp] - want)) <= 1e-11 * sc, (call, p)


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    # m = 81 is the first order whose work matrices leave shared memory:
    # 4 * 81^2 * 41 = 1,076,004 doubles > 1,048,576 (m = 80 with 41 probes
    # runs, see above); m = 128 with 20 probes: 1,310,720.
    for m, nprobe in ((81, 41), (128, 20)):
        H = torch.zeros(nprobe * m * (m + 1), dtype=torch.float64, device="cuda")
        c = torch.zeros(nprobe * m, dtype=torch.float64, device="cuda")
        with pytest.raises(B.LogdetError) as e:
            B.logdet_hessenberg_log_e1_noalloc(H, m + 1, None, m, nprobe, c)
        assert e.value.code == B.EINVAL, (m, nprobe)
    with pytest.raises(B.LogdetError):
        B.logdet_hessenberg_log_e1_noalloc(H, m + 1, None, 8, 5000, c)
