"""Matrix-free gridded operators (logdet_create_grid): the Wendland covariance
of the GRF study (Sec. 4) applied by a convolution kernel.  Checks against the
explicit CSR of the same operator: the SpMM bit-exact on integer tables, the
Gershgorin interval, FP64 estimates against the oracle at the FP64 bar, the
mixed path against FP64, and the server / plan paths against the blocking
call (bit-identical)."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_07004_gb300 import binding as B  # noqa: E402

RTOL_FP64 = 1e-10


@pytest.mark.parametrize("nx,ny,R", [(37, 23, 3), (530, 9, 5), (600, 40, 12), (5, 4, 6)])
def test_grid_spmm_integer_bit_exact(nx, ny, R):
    # integer table (exact products and sums), ragged segments, radius larger
    # than the grid in the last case
    rng = np.random.default_rng(R)
    T = rng.integers(-3, 4, size=(R + 1, R + 1)).astype(np.float64)
    T[0, 0] = 200.0
    A = W.grid_operator_csr(nx, ny, T)
    b, ld = 7, 8
    X = np.zeros((A.n, ld))
    X[:, :b] = O.rademacher_block(2, 0, A.n, b)
    with B.Handle.grid(nx, ny, T) as h:
        n, nnz, lo, hi = h.info()
        y = torch.zeros(A.n * ld, dtype=torch.float64, device="cuda")
        h.spmm(torch.as_tensor(X.ravel(), device="cuda"), y, b, ld)
        got = y.view(A.n, ld).cpu().numpy()
    assert (n, nnz) == (A.n, A.nnz)
    assert np.array_equal(got, A.to_scipy() @ X)


def _wendland(nx, ny, theta, nugget):
    T = W.wendland_table(theta, nugget)
    return T, W.grid_operator_csr(nx, ny, T)


def test_grid_gershgorin_matches_oracle():
    T, A = _wendland(41, 33, 5.0, 0.1)
    with B.Handle.grid(41, 33, T) as h:
        _, _, lo, hi = h.info()
    olo, ohi = O.gershgorin_interval(A.to_scipy())
    assert lo == pytest.approx(olo, rel=1e-14, abs=1e-14)
    assert hi == pytest.approx(ohi, rel=1e-14)


@pytest.mark.parametrize("method,k", [("oslq", 0), ("osaiop", 4), ("osaiop", 8)])
def test_grid_fp64_parity(method, k):
    T, A = _wendland(45, 38, 4.5, 0.05)
    Q = A.to_scipy()
    with B.Handle.grid(45, 38, T) as h:
        if method == "oslq":
            est = O.oslq(Q, 24, 25, seed=2)
            res = h.oslq(24, 25, seed=2)
        else:
            est = O.osaiop(Q, 24, 20, k=k, seed=2)
            res = h.osaiop(24, 20, iop_window=k, seed=2)
    assert abs(res.logdet - est.logdet) <= RTOL_FP64 * abs(est.logdet)
    np.testing.assert_allclose(res.per_probe, est.per_probe, rtol=1e-9, atol=1e-9)


def test_grid_mixed_shift_server_and_plan():
    T, A = _wendland(70, 50, 6.0, 0.02)
    with B.Handle.grid(70, 50, T) as h:
        r64 = h.osaiop(30, 20, iop_window=4, seed=5, shift=0.01)
        r32 = h.osaiop(30, 20, iop_window=4, seed=5, shift=0.01, precision=B.MIXED_FP32)
        assert abs(r32.logdet - r64.logdet) <= 1e-4 * abs(r64.logdet)
        est = O.osaiop((A.to_scipy() + 0.01 * __import__("scipy").sparse.eye(A.n)).tocsr(),
                       30, 20, k=4, seed=5)
        assert abs(r64.logdet - est.logdet) <= RTOL_FP64 * abs(est.logdet)
        with B.Server(4 << 30) as srv:
            ids = [srv.submit(h, B.METHOD_OSLQ, 30, 20, seed=s) for s in range(3)]
            served = [srv.wait(i) for i in ids]
        with B.Plan(h, B.METHOD_OSLQ, 30, 20) as plan:
            replay = [plan.run(s) for s in range(3)]
        for s in range(3):
            want = h.oslq(30, 20, seed=s)
            assert served[s].logdet == want.logdet == replay[s].logdet
            assert np.array_equal(served[s].per_probe, want.per_probe)


def test_grid_invalid_arguments():
    T = W.wendland_table(3.0)
    with pytest.raises(B.LogdetError):
        B.Handle.grid(0, 5, T)
    with pytest.raises(B.LogdetError):
        B.Handle.grid(5, 5, np.zeros((98, 98)))   # radius 97 > 96
    bad = T.copy()
    bad[1, 1] = np.nan
    with pytest.raises(B.LogdetError):
        B.Handle.grid(5, 5, bad)
    with B.Handle.grid(10, 10, T) as h:
        with pytest.raises(B.LogdetError):
            h.oslq(9, 5, precision=B.MIXED_BF16VEC)
        with pytest.raises(B.LogdetError):
            h.osaiop(9, 5, precision=B.MIXED_F32X2)


def test_quadform_csr_and_grid():
    T, A = _wendland(33, 29, 4.0, 0.2)
    x = np.random.default_rng(0).standard_normal(A.n)
    Q = A.to_scipy()
    want = float(x @ (Q @ x) + 0.3 * x @ x)
    xd = torch.as_tensor(x, device="cuda")
    with B.Handle.grid(33, 29, T) as hg, B.Handle.from_csr(A) as hc:
        assert hg.quadform(xd, 0.3) == pytest.approx(want, rel=1e-13)
        assert hc.quadform(xd, 0.3) == pytest.approx(want, rel=1e-13)


def test_grf_loglik_sweep_recovers_theta():
    """GRF study on a 60 x 50 grid: field drawn with precision Q(6) (Wendland
    support 6 cells, nugget 0.1); the sweep over theta = 3..8 must assemble
    L(theta) from its log-determinants and quadratic forms, match the oracle
    for one theta at the FP64 bar, and peak at theta = 6 (the exact
    log-likelihood peaks there by >= 20 units, far above the estimator error)."""
    import math
    from paper_2606_07004_gb300 import grf
    nx, ny = 60, 50
    x = W.grf_sample(nx, ny, W.wendland_table(6.0, 0.1), seed=3)
    thetas = [3.0, 4.0, 5.0, 6.0, 7.0, 8.0]
    sw = grf.loglik_sweep(torch.as_tensor(x, device="cuda"), nx, ny, thetas, nugget=0.1,
                          num_probes=30, krylov_steps=30, precision=B.FP64, seed=1)
    n = nx * ny
    for ld, q, ll in zip(sw.logdet, sw.quad, sw.loglik):
        assert ll == pytest.approx(0.5 * ld - 0.5 * q - 0.5 * n * math.log(2 * math.pi), rel=1e-15)
    assert sw.theta_hat == 6.0
    A = W.grid_operator_csr(nx, ny, W.wendland_table(5.0, 0.1))
    est = O.osaiop(A.to_scipy(), 30, 30, k=2, seed=1, tol=1e-6)
    assert abs(sw.logdet[2] - est.logdet) <= RTOL_FP64 * abs(est.logdet)
    sign, exact = np.linalg.slogdet(A.to_scipy().toarray())
    assert abs(sw.logdet[2] - exact) <= 0.02 * abs(exact)
