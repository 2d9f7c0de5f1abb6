"""Pins for the FP64 CPU oracle, against facts that do not come from the oracle.

Each test names the passage of the paper whose arithmetic it fixes and what
mistake it would catch.  None of these need a GPU.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle as O
from oracle import estimators as E
from oracle import rademacher as R
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense_logm_sym(A):
    lam, U = np.linalg.eigh(A)
    return (U * np.log(lam)) @ U.T


# ---------------------------------------------------------------------------
# Probe spec (Algorithms 2 and 3: Rademacher sketch and residual probes)
# ---------------------------------------------------------------------------

def test_splitmix64_published_outputs():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    got = [int(x) for x in R.splitmix64_sequence(0, 3)]
    assert got == want


def test_rademacher_entry_is_counter_output():
    # Column c, row i of a stream is output number c*2^32 + i of the generator
    # seeded with the stream key: for column 0 that is the plain sequence.
    key = int(R.stream_key(7, 1))
    seq = R.splitmix64_sequence(key, 50)
    block = R.rademacher_block(7, 1, 50, 1)[:, 0]
    assert np.array_equal(block, np.where((seq >> np.uint64(63)) == 0, 1.0, -1.0))


def test_rademacher_statistics():
    n, N = 32, 20000
    G = R.rademacher_block(11, 1, n, N)
    assert set(np.unique(G)) == {-1.0, 1.0}
    assert abs(G.mean()) < 5.0 / math.sqrt(G.size)
    C = G @ G.T / N                      # E[g g^T] = I
    off = C - np.diag(np.diag(C))
    assert np.allclose(np.diag(C), 1.0)
    assert np.max(np.abs(off)) < 6.0 / math.sqrt(N)
    # streams and seeds are different draws
    assert not np.array_equal(R.rademacher_block(11, 0, n, 4), R.rademacher_block(11, 1, n, 4))
    assert not np.array_equal(R.rademacher_block(11, 0, n, 4), R.rademacher_block(12, 0, n, 4))


# ---------------------------------------------------------------------------
# Spectral interval (Sec. 2.1, Gershgorin; clamp R3)
# ---------------------------------------------------------------------------

def test_gershgorin_closed_forms():
    lo, hi = O.gershgorin_interval(W.laplacian_2d(9, shift=0.25).to_scipy())
    assert lo == pytest.approx(0.25, abs=1e-14) and hi == pytest.approx(8.25, abs=1e-14)
    lo, hi = O.gershgorin_interval(W.laplacian_3d(5, shift=0.5).to_scipy())
    assert lo == pytest.approx(0.5, abs=1e-14) and hi == pytest.approx(12.5, abs=1e-14)
    lo, hi = O.gershgorin_interval(W.matern_2d(8, 0.05).to_scipy())
    assert lo == pytest.approx(0.05**2 + 8 * 0.05 + 16 + 4 - (8 * 4.05 + 12), abs=1e-12)
    assert lo == pytest.approx(-23.9975, abs=1e-12) and hi == pytest.approx(64.8025, abs=1e-12)
    G = W.powerlaw_graph_laplacian(3000, seed=1).with_diagonal_shift(0.03)
    lo, hi = O.gershgorin_interval(G.to_scipy())
    deg = np.diff(G.rowptr) - 1
    assert lo == pytest.approx(0.03, abs=1e-12)
    assert hi == pytest.approx(2 * deg.max() + 0.03, abs=1e-9)


def test_gershgorin_brute_force_dense():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((12, 12))
    A = A + A.T
    Ad = np.abs(A)
    R_ = Ad.sum(axis=1) - np.diag(Ad)
    lo, hi = O.gershgorin_interval(sp.csr_matrix(A))
    assert lo == pytest.approx(float(np.min(np.diag(A) - R_)), rel=1e-14)
    assert hi == pytest.approx(float(np.max(np.diag(A) + R_)), rel=1e-14)


def test_spectral_interval_clamp():
    lo, hi = O.spectral_interval(W.matern_2d(8, 0.05).to_scipy())
    assert hi == pytest.approx(64.8025) and lo == pytest.approx(1e-6 * 64.8025)
    assert O.spectral_interval(None, lam=(0.5, 2.0)) == (0.5, 2.0)


# ---------------------------------------------------------------------------
# Lanczos + Gauss quadrature (Sec. 3.1, Eq. gauss_quadrature)
# ---------------------------------------------------------------------------

def test_gauss_quadrature_moment_exactness():
    # An m-point Gauss rule integrates t^p exactly for p <= 2m-1:
    # sum_k tau_k^2 theta_k^p = v^T J^p v / v^T v.  Catches wrong weights
    # (tau instead of tau^2), a dropped beta or an off-by-one in T.
    A = W.random_spd_dense_csr(40, seed=2, cond=50.0).to_scipy()
    J = A / 50.0
    v = np.random.default_rng(3).standard_normal(40)
    m = 6
    al, be = O.lanczos(J, v, m, reorth=True)
    qd = O.gauss_quadrature_log(al, be)
    Jd = J.toarray()
    w = v / np.linalg.norm(v)
    x = w.copy()
    for p in range(2 * m):
        want = float(w @ x)
        got = float(np.sum(qd.tau2 * qd.theta ** p))
        assert got == pytest.approx(want, rel=1e-10, abs=1e-13), p
        x = Jd @ x


def test_lanczos_full_dimension_equals_dense_log():
    A = W.random_spd_dense_csr(30, seed=4, cond=30.0).to_scipy()
    J = A / 31.0
    v = np.random.default_rng(1).standard_normal(30)
    al, be = O.lanczos(J, v, 30, reorth=True)
    got = O.gauss_quadrature_log(al, be).value
    w = v / np.linalg.norm(v)
    want = float(w @ _dense_logm_sym(J.toarray()) @ w)
    assert got == pytest.approx(want, rel=1e-11, abs=1e-12)


def test_lanczos_identity_breaks_down_exactly():
    Q = W.scaled_identity(25, 3.0).to_scipy()
    al, be = O.lanczos(Q / 3.0, np.ones(25), 10)
    assert al.size == 1 and be.size == 0 and al[0] == pytest.approx(1.0)
    est = O.oslq(Q, 9, 10, seed=0)
    assert est.logdet == pytest.approx(25 * math.log(3.0), rel=1e-14)


def test_lanczos_diagonal_exact_at_distinct_count():
    d = np.repeat([0.5, 1.0, 2.0, 3.5, 7.0], 10)
    Q = W.diagonal_matrix(d).to_scipy()
    v = np.random.default_rng(9).standard_normal(d.size)
    al, be = O.lanczos(Q, v, 5)
    got = O.gauss_quadrature_log(al, be).value
    w = v / np.linalg.norm(v)
    assert got == pytest.approx(float(np.sum(w**2 * np.log(d))), rel=1e-12)


def test_lanczos_recurrence_residual():
    # Without re-orthogonalisation the three-term relation J V_m = V_m T_m +
    # beta_m v_{m+1} e_m^T still holds to rounding.  Rebuilt here from alpha, beta.
    Q = W.laplacian_2d(10, shift=0.2).to_scipy()
    J = Q / 8.2
    v = np.random.default_rng(0).standard_normal(100)
    m = 12
    al, be = O.lanczos(J, v, m + 1)
    V = [v / np.linalg.norm(v)]
    vp = np.zeros(100)
    for j in range(m):
        w = J @ V[j] - al[j] * V[j] - (be[j - 1] * vp if j else 0)
        vp = V[j]
        V.append(w / be[j])
    Vm = np.stack(V[:m], 1)
    T = np.diag(al[:m]) + np.diag(be[:m - 1], 1) + np.diag(be[:m - 1], -1)
    res = J @ Vm - Vm @ T
    res[:, -1] -= be[m - 1] * V[m]
    assert np.max(np.abs(res)) < 1e-13


# ---------------------------------------------------------------------------
# Algorithm 1 (Arnoldi-IOP-LOG)
# ---------------------------------------------------------------------------

def test_iop_full_window_is_arnoldi():
    # k = m: each column orthogonalised against all previous ones (MGS
    # Arnoldi), so V is orthonormal and H = V^T Q~ V, Arnoldi relation exact.
    A = W.random_spd_dense_csr(60, seed=6, cond=100.0).to_scipy() / 10.0
    v = np.random.default_rng(2).standard_normal(60)
    run = O.arnoldi_iop(A, v, 15, k=15)
    V, H = run.V, run.H
    assert np.max(np.abs(V.T @ V - np.eye(15))) < 1e-12
    assert np.max(np.abs(V.T @ (A @ V) - H)) < 1e-12
    assert np.max(np.abs(np.tril(H, -2))) == 0.0


def test_iop_window_two_matches_lanczos():
    # For symmetric Q and k = 2, IOP is Lanczos: H is tridiagonal with
    # diag = alpha_j and subdiag = beta_j (independent code: lanczos()).
    Q = W.laplacian_2d(12, shift=0.3).to_scipy() / 3.0
    v = np.random.default_rng(4).standard_normal(Q.shape[0])
    run = O.arnoldi_iop(Q, v, 10, k=2)
    al, be = O.lanczos(Q, v, 11)
    assert np.allclose(np.diag(run.H), al[:10], rtol=1e-12, atol=1e-13)
    assert np.allclose(np.diag(run.H, -1), be[:9], rtol=1e-12)
    assert np.allclose(np.diag(run.H, 1), be[:9], rtol=1e-9)
    assert np.max(np.abs(np.triu(run.H, 2))) == 0.0


def test_iop_log_action_full_dimension_is_dense_logm():
    A = W.random_spd_dense_csr(20, seed=8, cond=40.0).to_scipy()
    lo, hi = float(np.linalg.eigvalsh(A.toarray())[0]), float(np.linalg.eigvalsh(A.toarray())[-1])
    gamma = math.sqrt(lo * hi)
    v = np.random.default_rng(5).standard_normal(20)
    y = O.iop_log_action(A / gamma, v, 20, 20, math.log(gamma))
    want = sla.logm(A.toarray()).real @ v
    assert np.allclose(y, want, rtol=1e-9, atol=1e-10)


def test_iop_logm_inverts_expm():
    Q = W.laplacian_2d(8, shift=0.5).to_scipy() / 3.0
    run = O.arnoldi_iop(Q, np.ones(64), 12, k=4)
    L = sla.logm(run.H)
    assert np.allclose(sla.expm(L), run.H, atol=1e-12)


def test_iop_tol_break_keeps_column():
    # Q~ = I: w = v_1 - (v_1^T v_1) v_1 = 0 at m = 1, so m_eff = 1 and H = [[1]].
    run = O.arnoldi_iop(sp.identity(10, format="csr"), np.ones(10), 5, k=2)
    assert run.m_eff == 1 and run.H.shape == (1, 1) and run.H[0, 0] == pytest.approx(1.0)


# ---------------------------------------------------------------------------
# Hutch++ split (Algorithms 2/3) and the assembly n log(alpha) + tr
# ---------------------------------------------------------------------------

def test_orth_properties():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((50, 6))
    A = O.orth(Y)
    assert np.allclose(A.T @ A, np.eye(6), atol=1e-14)
    assert np.allclose(A @ (A.T @ Y), Y, atol=1e-12)
    Y2 = np.concatenate([Y, Y[:, :2] @ np.array([[1.0], [2.0]])], axis=1)
    assert O.orth(Y2).shape[1] == 6
    # A dependent column in the middle: the basis must still span every column.
    Y3 = Y.copy()
    Y3[:, 2] = Y[:, 0] - 3.0 * Y[:, 1]
    A3 = O.orth(Y3)
    assert A3.shape[1] == 5
    assert np.allclose(A3.T @ A3, np.eye(5), atol=1e-14)
    assert np.allclose(A3 @ (A3.T @ Y3), Y3, atol=1e-12)


def _hadamard(n):
    H = np.array([[1.0]])
    while H.shape[0] < n:
        H = np.block([[H, H], [H, -H]])
    return H


@pytest.mark.parametrize("method", ["oslq", "osaiop"])
def test_exact_with_hadamard_residual_probes(method):
    # With G a Hadamard matrix, (1/r) sum_j g_j g_j^T = I exactly, so the
    # residual term equals tr((I-P) L (I-P)); with m = n the Krylov parts are
    # exact too, hence the estimate is the exact log-determinant.  This pins
    # the 1/r weight, the ||z||^2 factor, the projection, n log(alpha) and,
    # for OSA-IOP, the log(gamma/alpha) shift.
    A = W.laplacian_2d(4, shift=0.5).to_scipy()
    n = 16
    S = O.rademacher_block(3, 0, n, 3)
    G = _hadamard(n)
    exact = np.linalg.slogdet(A.toarray())[1]
    if method == "oslq":
        est = O.oslq(A, 0 + 3 * 3, n, S=S, G=G, reorth=True)
    else:
        est = O.osaiop(A, 9, n, k=n, S=S, G=G)
    assert est.r == n
    assert est.logdet == pytest.approx(exact, rel=1e-10)


@pytest.mark.parametrize("method", ["oslq", "osaiop"])
def test_full_sketch_recovers_exact(method):
    # s >= n: A spans R^n, every z_j = 0 and the subspace part is the trace.
    Q = W.laplacian_2d(3, shift=1.0).to_scipy()
    n = 9
    exact = np.linalg.slogdet(Q.toarray())[1]
    if method == "oslq":
        est = O.oslq(Q, 3 * n + 2, n, seed=1, reorth=True)
    else:
        est = O.osaiop(Q, 3 * n + 2, n, k=n, seed=1)
    assert est.s_eff == n
    assert np.allclose(est.z_norm2, 0.0, atol=1e-20)
    assert est.logdet == pytest.approx(exact, rel=1e-10)


@pytest.mark.parametrize("method", ["oslq", "osaiop"])
def test_scale_invariance(method):
    # log det(cQ) = log det Q + n log c with the same probes: alpha and gamma
    # scale with c, the scaled operators do not change.
    Q = W.laplacian_2d(10, shift=0.2).to_scipy()
    c = 7.5
    f = (lambda M: O.oslq(M, 9, 15, seed=2)) if method == "oslq" else \
        (lambda M: O.osaiop(M, 9, 15, k=2, seed=2))
    a, b = f(Q), f(c * Q)
    assert b.logdet - a.logdet == pytest.approx(100 * math.log(c), rel=1e-11)


@pytest.mark.parametrize("method", ["oslq", "osaiop"])
def test_permutation_invariance(method):
    A = W.laplacian_2d(7, shift=0.4)
    n = A.n
    perm = np.random.default_rng(3).permutation(n)
    Ap = W.permute_symmetric(A, perm)
    S = O.rademacher_block(1, 0, n, 3)
    G = O.rademacher_block(1, 1, n, 4)
    f = O.oslq if method == "oslq" else (lambda *a, **k: O.osaiop(*a, k=2, **k))
    e1 = f(A.to_scipy(), 10, 12, S=S, G=G)
    e2 = f(Ap.to_scipy(), 10, 12, S=S[perm], G=G[perm])
    assert e2.logdet == pytest.approx(e1.logdet, rel=1e-12)


@pytest.mark.slow
@pytest.mark.parametrize("method", ["oslq", "osaiop"])
def test_unbiased_against_closed_form(method):
    # Hutch++ is unbiased; with m = 20 on a 12x12 grid the quadrature error is
    # negligible, so the mean over seeds must match the analytic log-det.
    Q = W.laplacian_2d(12, shift=0.3).to_scipy()
    exact = W.closed_form_logdet_laplacian_2d(12, shift=0.3)
    f = (lambda s: O.oslq(Q, 9, 20, seed=s)) if method == "oslq" else \
        (lambda s: O.osaiop(Q, 9, 20, k=2, seed=s))
    vals = np.array([f(s).logdet for s in range(200)])
    se = vals.std(ddof=1) / math.sqrt(vals.size)
    assert abs(vals.mean() - exact) < 4 * se + 1e-9 * abs(exact)


def test_config1_closed_form_and_band():
    A = W.laplacian_2d(64, shift=0.1)
    exact = W.closed_form_logdet_laplacian_2d(64, shift=0.1)
    assert exact == pytest.approx(5018.309092513560, rel=1e-13)
    assert exact == pytest.approx(np.linalg.slogdet(A.to_scipy().toarray())[1], rel=1e-12)
    est = O.oslq(A.to_scipy(), 30, 30, seed=0)
    assert abs(est.logdet - exact) / exact < 1e-2


def test_dense_cholesky_band():
    A = W.laplacian_3d(11, shift=0.05).to_scipy()
    exact = 2 * np.sum(np.log(np.diag(np.linalg.cholesky(A.toarray()))))
    for est in (O.oslq(A, 30, 40, seed=4), O.osaiop(A, 30, 40, k=4, seed=4)):
        assert abs(est.logdet - exact) / abs(exact) < 1e-2


def test_rounding_sensitivity_supports_1e10_tolerance():
    # Two summation orders (BLAS dot versus correctly rounded fsum) must agree
    # far inside the 1e-10 parity tolerance on the 64x64 FP64 workload.
    Q = W.laplacian_2d(64, shift=0.1).to_scipy()
    a = O.oslq(Q, 30, 30, seed=0)
    b = O.oslq(Q, 30, 30, seed=0, dot="fsum")
    assert abs(a.logdet - b.logdet) / abs(a.logdet) < 1e-12
    c = O.osaiop(Q, 12, 20, k=2, seed=0)
    d = O.osaiop(Q, 12, 20, k=2, seed=0, dot="fsum")
    assert abs(c.logdet - d.logdet) / abs(c.logdet) < 1e-12


def test_mgs_window_versus_classical_gram_schmidt():
    # Reading R5 fixes MGS order; a one-pass (classical) window differs only by
    # rounding on these operators.  Implemented inline from Algorithm 1 with the
    # window dots taken before any subtraction.
    Q = W.laplacian_3d(12, shift=0.01).to_scipy()
    lo, hi = O.spectral_interval(Q)
    gamma = math.sqrt(lo * hi)
    Qt = Q / gamma
    v = O.rademacher_block(0, 0, Q.shape[0], 1)[:, 0]
    for k in (2, 4, 8):
        run = O.arnoldi_iop(Qt, v, 30, k=k)
        V = [v / np.linalg.norm(v)]
        Hc = np.zeros((31, 30))
        for m in range(30):
            w = Qt @ V[m]
            js = range(max(0, m - k + 1), m + 1)
            c = [float(V[j] @ w) for j in js]
            for j, cj in zip(js, c):
                Hc[j, m] = cj
                w = w - cj * V[j]
            h = np.linalg.norm(w)
            Hc[m + 1, m] = h
            V.append(w / h)
        c1, _ = E.principal_logm_e1(run.H)
        c2, _ = E.principal_logm_e1(Hc[:30, :30])
        assert np.max(np.abs(c1 - c2)) < 1e-11


def test_scaling_makes_log_operator_semidefinite():
    # Sec. 3.2: with alpha = lambda_max bound, J = Q/alpha has spectrum in
    # (0, 1], so every quadrature K(q) = q^T log(J) q is <= 0.  Sec. 2.2: with
    # alpha = lambda_min bound, L = log(Q/alpha) is PSD, so every q^T L q >= 0.
    # A wide spectrum (kappa ~ 1e3) makes any other alpha produce both signs.
    Q = W.laplacian_2d(20, shift=0.01).to_scipy()
    a = O.oslq(Q, 30, 25, seed=5)
    assert np.all(a.per_probe <= 0.0)
    lo, hi = O.gershgorin_interval(Q)
    assert a.log_alpha == pytest.approx(math.log(hi), rel=1e-15)
    b = O.osaiop(Q, 30, 25, k=2, seed=5)
    assert np.all(b.per_probe >= 0.0)
    assert b.log_alpha == pytest.approx(math.log(lo), rel=1e-15)


def test_gaussian_probes_statistics_and_definition():
    from oracle.rademacher import gaussian_block, rademacher_bits, splitmix64_mix
    G = gaussian_block(4, 1, 64, 4000)
    assert abs(G.mean()) < 5 / math.sqrt(G.size)
    assert abs(G.var() - 1.0) < 0.02
    assert abs(np.mean(G ** 4) - 3.0) < 0.1                 # normal kurtosis
    z = int(rademacher_bits(4, 1, 1, 1)[0, 0])
    w = int(splitmix64_mix(np.uint64(z)))
    u1 = ((z >> 11) + 1) * 2.0 ** -53
    u2 = (w >> 11) * 2.0 ** -53
    assert G[0, 0] == pytest.approx(math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2), rel=1e-15)


@pytest.mark.parametrize("method", ["oslq", "osaiop"])
def test_plain_slq_is_hutchinson_with_gauss_rules(method):
    # hutchpp=False: logdet = n log alpha + (1/r) sum_j |g_j|^2 K(g_j); with
    # Hadamard probes (1/r) G G^T = I and m = n that is the exact log det.
    A = W.laplacian_2d(4, shift=0.5).to_scipy()
    G = _hadamard(16)
    exact = np.linalg.slogdet(A.toarray())[1]
    if method == "oslq":
        est = O.oslq(A, 16, 16, G=G, hutchpp=False, reorth=True)
    else:
        est = O.osaiop(A, 16, 16, k=16, G=G, hutchpp=False)
    assert est.s == 0 and est.r == 16
    assert est.logdet == pytest.approx(exact, rel=1e-10)
    # and it is unbiased over seeds with Rademacher probes
    Q = W.laplacian_2d(10, shift=0.3).to_scipy()
    vals = [O.oslq(Q, 6, 20, seed=s, hutchpp=False).logdet for s in range(150)]
    exact = W.closed_form_logdet_laplacian_2d(10, shift=0.3)
    assert abs(np.mean(vals) - exact) < 4 * np.std(vals) / math.sqrt(len(vals))


def test_paper_tolerance_mode_stops_probes_early():
    # tol = 1e-6 (the GRF experiment's setting) on Q = diag with 4 distinct
    # values: every Krylov run stops at dimension 4 with exact forms, and with
    # Hadamard residual probes the whole estimate is the exact log det.
    d = np.repeat([1.0, 2.0, 4.0, 8.0], 16)
    Q = W.diagonal_matrix(d).to_scipy()
    v = np.random.default_rng(0).standard_normal(64)
    run = O.arnoldi_iop(Q / 2.0, v, 20, k=2, tol=1e-6)
    assert run.m_eff == 4
    al, be = O.lanczos(Q / 8.0, v, 20, tol=1e-6)
    assert al.size == 4
    S = O.rademacher_block(1, 0, 64, 3)
    G = _hadamard(64)
    exact = float(np.sum(np.log(d)))
    assert O.osaiop(Q, 9, 20, k=2, S=S, G=G, tol=1e-6).logdet == pytest.approx(exact, rel=1e-10)
    assert O.oslq(Q, 9, 20, S=S, G=G, tol=1e-6).logdet == pytest.approx(exact, rel=1e-10)


# ---------------------------------------------------------------------------
# Spectral interval above n = 20000, where spectral_interval switches from the
# row loop to the vectorised sums (Sec. 2.1, Gershgorin; clamp R3).  Every
# full-size oracle run takes that branch.
# ---------------------------------------------------------------------------

LARGE_CLOSED_FORMS = [
    # (matrix, its Gershgorin interval from the stencil's row sums)
    ("lap2d_151x149", lambda: W.laplacian_2d(151, 149, shift=0.3), 0.3, 8.3),
    ("lap3d_31x29x27", lambda: W.laplacian_3d(31, 29, 27, shift=0.02), 0.02, 12.02),
    # (k2 + 4)^2 + 4 on the diagonal; off-diagonal |.| sums to 8 (k2 + 4) + 4 + 8
    ("matern_150", lambda: W.matern_2d(150, 0.05), -23.9975, 64.8025),
]


@pytest.mark.parametrize("name,make,lo,hi", LARGE_CLOSED_FORMS, ids=[c[0] for c in LARGE_CLOSED_FORMS])
def test_gershgorin_fast_closed_forms(name, make, lo, hi):
    A = make()
    assert A.n > 20000
    glo, ghi = E._gershgorin_fast(A.to_scipy())
    assert glo == pytest.approx(lo, abs=1e-12) and ghi == pytest.approx(hi, abs=1e-12)
    # the branch spectral_interval takes at this size, with the clamp (R3)
    slo, shi = O.spectral_interval(A.to_scipy())
    assert shi == pytest.approx(hi, abs=1e-12)
    assert slo == pytest.approx(lo if lo > 0 else 1e-6 * hi, rel=1e-12)


def test_gershgorin_fast_full_size_workloads():
    # The 128^3 Laplacian + 0.01 I and the 1024^2 Matern operator at the
    # sizes the benchmark's oracle baseline runs.
    lo, hi = E._gershgorin_fast(W.laplacian_3d(128, shift=0.01).to_scipy())
    assert lo == pytest.approx(0.01, abs=1e-13) and hi == pytest.approx(12.01, abs=1e-13)
    lo, hi = E._gershgorin_fast(W.matern_2d(1024, 0.05).to_scipy())
    assert lo == pytest.approx(-23.9975, abs=1e-12) and hi == pytest.approx(64.8025, abs=1e-12)


def test_gershgorin_fast_power_law_graph():
    # L + s I of a graph with unit weights: row i has diagonal deg_i + s and
    # off-diagonal sum deg_i, so the interval is [s, 2 max deg + s].
    G = W.powerlaw_graph_laplacian(30000, seed=2).with_diagonal_shift(0.07)
    deg = np.diff(G.rowptr) - 1
    lo, hi = E._gershgorin_fast(G.to_scipy())
    assert lo == pytest.approx(0.07, abs=1e-12)
    assert hi == pytest.approx(2 * deg.max() + 0.07, abs=1e-9)


def test_gershgorin_fast_brute_force_random_signs():
    # Random symmetric matrix with mixed signs, rows of 1 to ~60 entries, an
    # empty row and a row without its diagonal, against row sums of |Q| formed
    # by a sparse product (an independent evaluation of the same definition).
    rng = np.random.default_rng(17)
    n = 25000
    nnz = 400000
    r = rng.integers(0, n, nnz)
    c = np.minimum(r + rng.geometric(0.02, nnz), n - 1)
    v = rng.standard_normal(nnz)
    U = sp.coo_matrix((v, (r, c)), shape=(n, n)).tocsr()
    D = sp.diags(rng.standard_normal(n) * 30.0)
    Q = (U + U.T + D).tocsr()
    Q = Q.tolil()
    Q[123, :] = 0.0                      # empty row (and column)
    Q[:, 123] = 0.0
    Q[4567, 4567] = 0.0                  # row without a stored diagonal
    Q = Q.tocsr()
    Q.eliminate_zeros()
    Q.sort_indices()
    assert Q.indptr[124] == Q.indptr[123]
    diag = Q.diagonal()
    R_ = np.asarray(abs(Q) @ np.ones(n)).ravel() - np.abs(diag)
    want_lo, want_hi = float(np.min(diag - R_)), float(np.max(diag + R_))
    lo, hi = E._gershgorin_fast(Q)
    assert lo == pytest.approx(want_lo, rel=1e-13) and hi == pytest.approx(want_hi, rel=1e-13)


def test_gershgorin_fast_equals_row_loop():
    # The vectorised sums and the row loop are the same sums in different
    # orders: equal to a few units in the last place.
    for A in (W.laplacian_2d(151, 149, shift=0.3), W.laplacian_3d(31, 29, 27, shift=0.02),
              W.matern_2d(150, 0.05)):
        Qs = A.to_scipy()
        Qs.data = Qs.data * (1.0 + 0.01 * np.sin(np.arange(Qs.nnz)))   # distinct values
        assert E._gershgorin_fast(Qs) == pytest.approx(O.gershgorin_interval(Qs), rel=1e-14)


# ---------------------------------------------------------------------------
# Degenerate spectra: a non-positive Ritz value (Sec. 3.1 Gauss rule, R17) and
# a Hessenberg matrix whose principal logarithm is not real (Algorithm 1, R16)
# ---------------------------------------------------------------------------

def test_gauss_rule_clamps_nonpositive_ritz_value():
    # T = [[1/2, 1], [1, 1/2]] has eigenvalues -1/2 and 3/2 with eigenvectors
    # (1, -1)/sqrt 2 and (1, 1)/sqrt 2, so both weights are 1/2.
    qd = O.gauss_quadrature_log([0.5, 0.5], [1.0], clamp=1e-3)
    assert qd.nonpositive
    assert np.allclose(np.sort(qd.theta), [1e-3, 1.5], rtol=1e-14)
    assert np.allclose(qd.tau2, [0.5, 0.5], rtol=1e-14)
    assert qd.value == pytest.approx(0.5 * math.log(1e-3) + 0.5 * math.log(1.5), rel=1e-14)
    ok = O.gauss_quadrature_log([2.0, 2.0], [1.0])          # eigenvalues 1 and 3
    assert not ok.nonpositive
    assert ok.value == pytest.approx(0.5 * math.log(3.0), rel=1e-14)


def test_oslq_indefinite_diagonal_clamps_to_lower_bound():
    # Q = diag(-1 (a times), 2 (n - a times)): Gershgorin [-1, 2], clamped
    # lambda_lo = 2e-6 (R3), alpha = 2, J has eigenvalues -1/2 and 1.  Two
    # Lanczos steps from a +-1 probe g give theta = {-1/2, 1} with weights
    # a/n and (n-a)/n; -1/2 is clamped to lambda_lo/alpha = 1e-6 (R17), so
    # K(g) = (a/n) log(1e-6) and, without the Hutch++ split,
    # log det = n log 2 + (1/r) sum_j |g_j|^2 K(g_j) = n log 2 + a log(1e-6).
    n, a = 30, 7
    Q = W.diagonal_matrix(np.r_[np.full(a, -1.0), np.full(n - a, 2.0)]).to_scipy()
    est = O.oslq(Q, 5, 2, seed=3, hutchpp=False)
    assert est.flags & E.FLAG_NONPOSITIVE_RITZ
    assert est.logdet == pytest.approx(n * math.log(2.0) + a * math.log(1e-6), rel=1e-12)
    assert np.allclose(est.per_probe, (a / n) * math.log(1e-6), rtol=1e-12)
    spd = O.oslq(W.diagonal_matrix(np.r_[np.full(a, 1.0), np.full(n - a, 2.0)]).to_scipy(),
                 5, 2, seed=3, hutchpp=False)
    assert not spd.flags & E.FLAG_NONPOSITIVE_RITZ


def test_principal_logm_flags_negative_eigenvalue():
    # An eigenvalue on the negative real axis has no real logarithm:
    # log(-1) = i pi.  Upper triangular H = [[-1, 1/2], [0, 2]].
    c, ok = E.principal_logm_e1(np.array([[-1.0, 0.5], [0.0, 2.0]]))
    assert not ok
    assert c == pytest.approx([0.0, 0.0], abs=1e-12)       # real part of (i pi, 0)
    c, ok = E.principal_logm_e1(np.array([[1.0, 0.5], [0.0, 2.0]]))
    assert ok
    # log of [[1, b], [0, 2]] has first column (log 1, 0)
    assert c == pytest.approx([0.0, 0.0], abs=1e-14)
    c, ok = E.principal_logm_e1(np.array([[2.0, 0.0], [0.5, 1.0]]))
    assert ok
    # lower triangular [[l1, 0], [b, l2]]: (log A)_21 = b (log l1 - log l2)/(l1 - l2)
    assert c == pytest.approx([math.log(2.0), 0.5 * math.log(2.0)], rel=1e-13)


def test_osaiop_indefinite_sets_complex_log_flag():
    # Q = diag(-1, 2): gamma = sqrt(2e-6 * 2), the Hessenberg matrix of every
    # probe has the eigenvalue -1/gamma, so its principal log is not real.
    n, a = 24, 5
    Q = W.diagonal_matrix(np.r_[np.full(a, -1.0), np.full(n - a, 2.0)]).to_scipy()
    assert O.osaiop(Q, 6, 2, k=2, seed=1).flags & E.FLAG_COMPLEX_LOG
    spd = W.diagonal_matrix(np.r_[np.full(a, 1.0), np.full(n - a, 2.0)]).to_scipy()
    assert not O.osaiop(spd, 6, 2, k=2, seed=1).flags & E.FLAG_COMPLEX_LOG


def test_iop_window_amplifies_rounding_on_ill_conditioned_graph():
    # The batched irregular regime (power-law graph Laplacian + 3.84e-3 I,
    # kappa ~ 1e5; Algorithm 1 with window k = 4): one FP32 rounding of the
    # first Krylov vector changes the quadratic form z^T L z by more than
    # 5e-6 (relative) after m = 100 steps, by less than 1e-7 after m = 40.
    # Once Ritz values converge the incomplete orthogonalisation lets early
    # rounding grow, so at m = 100 no implementation with FP32 vectors can
    # follow the FP64 result to 1e-4 for small shifts (the tolerance of the
    # mixed path there is set by this, not by the kernels).
    n, sigma = 2 ** 15, 3.84e-3
    L = W.powerlaw_graph_laplacian(n, exponent=2.3, mean_degree=8.0, seed=7).to_scipy()
    Q = (L + sigma * sp.identity(n, format="csr")).tocsr()
    lo, hi = O.spectral_interval(Q)
    g = math.sqrt(lo * hi)
    Qt = Q / g
    z = O.rademacher_block(0, 1, n, 1)[:, 0]

    class RoundFirst:              # Q~ whose first product is rounded to FP32
        shape = Qt.shape

        def __init__(self):
            self.calls = 0

        def __matmul__(self, x):
            self.calls += 1
            y = Qt @ x
            return y.astype(np.float32).astype(np.float64) if self.calls == 1 else y

    for m, lo_bound, hi_bound in ((100, 5e-6, 1.0), (40, 0.0, 1e-7)):
        a = float(z @ O.iop_log_action(Qt, z, m, 4, math.log(g / lo)))
        b = float(z @ O.iop_log_action(RoundFirst(), z, m, 4, math.log(g / lo)))
        assert lo_bound < abs(a - b) / abs(a) < hi_bound, m
