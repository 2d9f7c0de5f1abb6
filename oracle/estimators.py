"""OSLQ and OSA-IOP, literally, in FP64 NumPy/SciPy (test infrastructure only).

Section / equation references are to the paper (arXiv 2606.07004):

* Sec. 2.1 (Algorithm 1, Arnoldi-IOP-LOG): the action log(Q)v through a
  Krylov basis built with an incomplete-orthogonalisation window, after the
  shift-scale Q~ = Q/gamma with gamma = sqrt(lambda_min * lambda_max)
  (Proposition 2.1).
* Sec. 2.2 (Algorithm 2, OSA-IOP): Hutch++ on L = log(Q/alpha) with
  alpha a lower spectral bound, log det Q = n log alpha + tr(L).
* Sec. 3.1 (Gauss quadrature): v^T f(Q) v ~ sum_k tau_k^2 f(theta_k) from the
  eigenpairs of the Lanczos tridiagonal T_m, tau_k = e_1^T u_k.
* Sec. 3.2-3.3 (Algorithm 3, OSLQ): J = Q/alpha with alpha = lambda_max,
  Y = J S, A = orth(Y); tr(log J) = sum_i K(q_i) + (1/r) sum_j ||z_j||^2 K(z_j/||z_j||)
  with z_j = (I - A A^T) g_j; log det Q = n log alpha + tr(log J).

Readings of silent or garbled passages (each one is also listed in the design
notes of the repository):

R1  OSLQ always scales J = Q/alpha with alpha = the Gershgorin upper bound;
    log det = n log alpha + tr(log J) is then exact algebra (Eq. scaled J).
R2  OSA-IOP: alpha = the lower spectral bound of Q and the shift
    log(gamma/alpha) I is always applied, so L = log(Q/alpha) (Eq. for L).
R3  A non-positive Gershgorin lower bound is replaced by 1e-6 * upper bound.
R4  OSLQ uses plain three-term Lanczos without re-orthogonalisation
    (``reorth=True`` exists only for the exactness pins).
R5  The IOP window has length k: column m is orthogonalised against
    v_i, i = max(1, m-k+1) .. m, in ascending (modified Gram-Schmidt) order.
R6  ``tol``: IOP stops when h_{m+1,m} < tol (the column m is kept); Lanczos
    truncates T to j x j when beta_j <= tol.
R7  OSA-IOP quadratic forms are q^T (L q) with L q from Algorithm 1.
R8  The sketch of Algorithm 2, written as log(L) S (garbled), is Y = L S.
R9  s = floor(m_vec/3) sketch columns, r = m_vec - 2 s residual probes, and
    the residual weight is 1/r (3/m_vec when 3 divides m_vec).
R11 The residual sum is tr_res = (1/r) sum_j ||z_j||^2 K(z_j/||z_j||); the
    factor in the printed loop of Algorithm 3 is applied once, not per term.
R13 Probes come from the SplitMix64 spec in ``rademacher.py``.
R14 orth(Y) is the thin QR factor with diag(R) > 0; a column whose |R_ii| is
    at most 1e-6 * max_j ||y_j|| is dropped (rank-deficient sketch).
R15 A residual probe with ||z_j|| = 0 contributes 0.
R16 log(H_m) is the principal matrix logarithm (scipy.linalg.logm); an H_m
    whose logarithm is not real (an eigenvalue on the negative real axis) sets
    FLAG_COMPLEX_LOG and its real part is used.
R17 A Ritz value theta <= 0 (an indefinite T_m) sets FLAG_NONPOSITIVE_RITZ and
    is clamped to lambda_lo / alpha, the lower spectral bound of J (Sec. 2.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .rademacher import gaussian_block, rademacher_block

CLAMP_REL = 1e-6       # R3
RANK_TOL = 1e-6        # R14
DEFAULT_TOL = 1e-12    # R6 default (absolute; the scaled operators are O(1))


def _dot_numpy(a, b):
    return float(np.dot(a, b))


def _dot_fsum(a, b):
    """Correctly rounded dot product (math.fsum over the exact-ish products)."""
    return math.fsum((np.asarray(a) * np.asarray(b)).tolist())


DOTS = {"numpy": _dot_numpy, "fsum": _dot_fsum}


# ---------------------------------------------------------------------------
# Spectral interval (Sec. 2.1, last paragraph before Algorithm 1)
# ---------------------------------------------------------------------------

def gershgorin_interval(Q: sp.csr_matrix) -> tuple[float, float]:
    """[min_i (a_ii - R_i), max_i (a_ii + R_i)], R_i = sum_{j != i} |a_ij|.

    R_i is summed in CSR (column) order, one row at a time.
    """
    Q = sp.csr_matrix(Q)
    lo, hi = math.inf, -math.inf
    indptr, indices, data = Q.indptr, Q.indices, Q.data
    n = Q.shape[0]
    for i in range(n):
        d = 0.0
        R = 0.0
        for p in range(indptr[i], indptr[i + 1]):
            if indices[p] == i:
                d = float(data[p])
            else:
                R += abs(float(data[p]))
        lo = min(lo, d - R)
        hi = max(hi, d + R)
    return lo, hi


def _gershgorin_fast(Q: sp.csr_matrix) -> tuple[float, float]:
    """Vectorised form of the same sums, for large n.  NumPy's segment reduction
    adds a row's entries in its own order, so the bounds can differ from the
    row loop's in the last bits."""
    Q = sp.csr_matrix(Q)
    n = Q.shape[0]
    rows = np.repeat(np.arange(n), np.diff(Q.indptr))
    is_d = Q.indices == rows
    d = np.zeros(n)
    d[rows[is_d]] = Q.data[is_d]
    off = np.where(is_d, 0.0, np.abs(Q.data))
    R = np.add.reduceat(off, Q.indptr[:-1]) if Q.nnz else np.zeros(n)
    R[np.diff(Q.indptr) == 0] = 0.0
    return float((d - R).min()), float((d + R).max())


def spectral_interval(Q, lam=None) -> tuple[float, float]:
    """(lambda_lo, lambda_hi): caller bounds if given, else clamped Gershgorin (R3)."""
    if lam is not None:
        return float(lam[0]), float(lam[1])
    Q = sp.csr_matrix(Q)
    lo, hi = _gershgorin_fast(Q) if Q.shape[0] > 20000 else gershgorin_interval(Q)
    if not hi > 0:
        raise ValueError("Gershgorin upper bound is not positive: matrix is not SPD")
    if not lo > 0:
        lo = CLAMP_REL * hi
    return lo, hi


# ---------------------------------------------------------------------------
# Lanczos tridiagonalisation and Gauss quadrature (Sec. 3.1)
# ---------------------------------------------------------------------------

def lanczos(J, q, m: int, tol: float = DEFAULT_TOL, reorth: bool = False, dot="numpy"):
    """m steps of symmetric Lanczos on J from q/||q||.

    Step j:  w = J v_j;  alpha_j = v_j^T w;  w = w - alpha_j v_j - beta_{j-1} v_{j-1};
             beta_j = ||w||;  v_{j+1} = w / beta_j.
    Returns (alpha[0:m_eff], beta[0:m_eff-1]).
    """
    dotf = DOTS[dot] if isinstance(dot, str) else dot
    v = np.asarray(q, dtype=np.float64)
    v = v / math.sqrt(dotf(v, v))
    v_prev = np.zeros_like(v)
    beta_prev = 0.0
    alphas, betas = [], []
    basis = [v] if reorth else None
    for j in range(m):
        w = J @ v
        a = dotf(v, w)
        alphas.append(a)
        if j == m - 1:
            break
        w = w - a * v - beta_prev * v_prev
        if reorth:  # full re-orthogonalisation, twice (exactness pins only)
            for _ in range(2):
                for u in basis:
                    w = w - dotf(u, w) * u
        b = math.sqrt(dotf(w, w))
        if b <= tol:
            break
        betas.append(b)
        v_prev, v = v, w / b
        beta_prev = b
        if reorth:
            basis.append(v)
    return np.array(alphas), np.array(betas)


@dataclass
class Quadrature:
    value: float            # sum_k tau_k^2 log(theta_k)
    theta: np.ndarray
    tau2: np.ndarray
    nonpositive: bool       # a Ritz value <= 0 was met (clamped)


def gauss_quadrature_log(alphas, betas, clamp: float | None = None) -> Quadrature:
    """e_1^T log(T_m) e_1 = sum_k tau_k^2 log(theta_k)  (Eq. gauss_quadrature).

    The weights are tau_k^2 with tau_k the first component of the unit
    eigenvector u_k of T_m.
    """
    alphas = np.asarray(alphas, dtype=np.float64)
    betas = np.asarray(betas, dtype=np.float64)
    if alphas.size == 1:
        theta = alphas.copy()
        U = np.ones((1, 1))
    else:
        theta, U = sla.eigh_tridiagonal(alphas, betas)
    tau2 = U[0, :] ** 2
    bad = bool(np.any(theta <= 0))
    if bad:
        theta = np.maximum(theta, clamp if clamp is not None else np.finfo(float).tiny)
    return Quadrature(float(np.sum(tau2 * np.log(theta))), theta, tau2, bad)


# ---------------------------------------------------------------------------
# Algorithm 1: Arnoldi with an incomplete-orthogonalisation window, log action
# ---------------------------------------------------------------------------

@dataclass
class IOPRun:
    V: np.ndarray       # n x m_eff, columns v_1..v_m
    H: np.ndarray       # m_eff x m_eff upper Hessenberg
    h_next: float       # h_{m+1,m}
    m_eff: int
    v_norm: float       # ||v|| of the starting vector


def arnoldi_iop(Qt, v, m_max: int, k: int = 2, tol: float = DEFAULT_TOL, dot="numpy") -> IOPRun:
    """Algorithm 1's basis loop with window k (R5, R6).

    Column m (1-based) of H: w = Q~ v_m; for j = max(1, m-k+1) .. m ascending:
    H[j, m] = v_j^T w;  w = w - H[j, m] v_j.  Then h = ||w||, H[m+1, m] = h;
    stop if h < tol (keeping column m), else v_{m+1} = w / h.
    """
    dotf = DOTS[dot] if isinstance(dot, str) else dot
    v = np.asarray(v, dtype=np.float64)
    vn = math.sqrt(dotf(v, v))
    V = [v / vn]
    H = np.zeros((m_max + 1, m_max))
    m_eff = 0
    h = math.inf
    for m in range(m_max):          # m is the 0-based column index
        w = Qt @ V[m]
        for j in range(max(0, m - k + 1), m + 1):
            H[j, m] = dotf(V[j], w)
            w = w - H[j, m] * V[j]
        h = math.sqrt(dotf(w, w))
        H[m + 1, m] = h
        m_eff = m + 1
        if h < tol:
            break
        if m + 1 < m_max:
            V.append(w / h)
    Vm = np.stack(V[:m_eff], axis=1)
    return IOPRun(Vm, H[:m_eff, :m_eff].copy(), float(h), m_eff, vn)


def principal_logm_e1(Hm: np.ndarray) -> tuple[np.ndarray, bool]:
    """First column of the principal logarithm of H_m (R16)."""
    Lm = sla.logm(Hm)
    ok = True
    if np.iscomplexobj(Lm):
        if np.max(np.abs(Lm.imag)) > 1e-10 * max(1.0, np.max(np.abs(Lm.real))):
            ok = False
        Lm = Lm.real
    return np.asarray(Lm[:, 0], dtype=np.float64), ok


def iop_log_action(Qt, v, m_max: int, k: int, shift: float, tol: float = DEFAULT_TOL,
                   dot="numpy", report: list | None = None) -> np.ndarray:
    """y = ||v|| V_m log(H_m) e_1 + shift * v  (Algorithm 1's return line with the
    constant term generalised: shift = log(gamma) gives log(Q) v, shift =
    log(gamma/alpha) gives L v of Sec. 2.2).  If ``report`` is a list, False is
    appended to it when log(H_m) is not real (R16)."""
    v = np.asarray(v, dtype=np.float64)
    if not np.any(v):
        return np.zeros_like(v)
    run = arnoldi_iop(Qt, v, m_max, k, tol, dot)
    c, ok = principal_logm_e1(run.H)
    if report is not None and not ok:
        report.append(False)
    return run.v_norm * (run.V @ c) + shift * v


# ---------------------------------------------------------------------------
# Hutch++ pieces
# ---------------------------------------------------------------------------

def orth(Y: np.ndarray) -> np.ndarray:
    """Orthonormal basis of span(Y) (R14): the thin QR factor, diag(R) > 0, of Y
    with its numerically dependent columns removed.  Columns are taken left to
    right; column j is dependent when the R_jj of the QR of the kept columns
    plus column j is at most RANK_TOL * max_i |y_i|."""
    Y = np.asarray(Y, dtype=np.float64)
    if Y.shape[1] == 0:
        return Y
    ref = float(np.max(np.linalg.norm(Y, axis=0)))
    Qf, R = np.linalg.qr(Y, mode="reduced")
    if R.shape[0] == Y.shape[1] and np.all(np.abs(np.diag(R)) > RANK_TOL * ref):
        return Qf * np.sign(np.diag(R))[None, :]        # full rank: one QR suffices
    kept = []
    for j in range(Y.shape[1]):
        _, R = np.linalg.qr(Y[:, kept + [j]], mode="reduced")
        if R.shape[0] > len(kept) and abs(R[len(kept), len(kept)]) > RANK_TOL * ref:
            kept.append(j)
    Qf, R = np.linalg.qr(Y[:, kept], mode="reduced")
    return Qf * np.sign(np.diag(R))[None, :]


def _split(num_probes: int) -> tuple[int, int]:
    if num_probes < 3:
        raise ValueError("num_probes must be >= 3")
    s = num_probes // 3
    return s, num_probes - 2 * s


@dataclass
class Estimate:
    logdet: float
    tr_sub: float
    tr_res: float
    log_alpha: float
    log_gamma: float
    s: int
    r: int
    s_eff: int
    per_probe: np.ndarray = field(default_factory=lambda: np.zeros(0))
    z_norm2: np.ndarray = field(default_factory=lambda: np.zeros(0))
    flags: int = 0


FLAG_NONPOSITIVE_RITZ = 1
FLAG_COMPLEX_LOG = 2
FLAG_RANK_DEFICIENT = 4


def _probes(n, s, r, seed, S, G, gaussian=False):
    gen = gaussian_block if gaussian else rademacher_block
    if S is None:
        S = gen(seed, 0, n, s)
    if G is None:
        G = gen(seed, 1, n, r)
    return np.asarray(S, dtype=np.float64), np.asarray(G, dtype=np.float64)


# ---------------------------------------------------------------------------
# Algorithm 3: OSLQ
# ---------------------------------------------------------------------------

def oslq(Q, num_probes: int, m: int, seed: int = 0, *, S=None, G=None, lam=None,
         tol: float = DEFAULT_TOL, reorth: bool = False, dot="numpy", hutchpp: bool = True,
         gaussian: bool = False) -> Estimate:
    """log det Q by Algorithm 3 with readings R1, R4, R6, R9, R11-R15.

    hutchpp=False is plain stochastic Lanczos quadrature (Hutchinson, Eq. TE
    with each quadratic form by the Gauss rule): no sketch, all num_probes
    probes residual (s = 0, r = num_probes).  gaussian=True draws N(0, 1)
    probes instead of +-1 (the alternative the paper allows for S)."""
    Q = sp.csr_matrix(Q, dtype=np.float64)
    n = Q.shape[0]
    lam_lo, lam_hi = spectral_interval(Q, lam)
    alpha = lam_hi                                   # R1
    clamp = lam_lo / alpha                           # R17
    J = sp.csr_matrix((Q.data / alpha, Q.indices, Q.indptr), shape=Q.shape)
    s, r = _split(num_probes) if hutchpp else (0, num_probes)
    if S is not None:
        s = S.shape[1]
    if G is not None:
        r = G.shape[1]
    S, G = _probes(n, s, r, seed, S, G, gaussian)
    flags = 0
    Y = J @ S                                        # Eq. power_sketch
    A = orth(Y)
    if A.shape[1] < s:
        flags |= FLAG_RANK_DEFICIENT
    per = []
    tr_sub = 0.0
    for i in range(A.shape[1]):                      # deterministic subspace part
        a_, b_ = lanczos(J, A[:, i], m, tol, reorth, dot)
        qd = gauss_quadrature_log(a_, b_, clamp)
        flags |= FLAG_NONPOSITIVE_RITZ if qd.nonpositive else 0
        per.append(qd.value)
        tr_sub += qd.value
    Z = G - A @ (A.T @ G)                            # z_j = (I - A A^T) g_j
    zn2 = np.einsum("ij,ij->j", Z, Z)
    tr_res = 0.0
    for j in range(Z.shape[1]):                      # stochastic residual part
        if zn2[j] == 0.0:                            # R15
            per.append(0.0)
            continue
        a_, b_ = lanczos(J, Z[:, j], m, tol, reorth, dot)
        qd = gauss_quadrature_log(a_, b_, clamp)
        flags |= FLAG_NONPOSITIVE_RITZ if qd.nonpositive else 0
        per.append(qd.value)
        tr_res += zn2[j] * qd.value
    tr_res /= r                                      # R9, R11
    logdet = n * math.log(alpha) + tr_sub + tr_res
    return Estimate(logdet, tr_sub, tr_res, math.log(alpha), 0.0, s, r, A.shape[1],
                    np.array(per), zn2, flags)


# ---------------------------------------------------------------------------
# Algorithm 2: OSA-IOP
# ---------------------------------------------------------------------------

def osaiop(Q, num_probes: int, m: int, k: int = 2, seed: int = 0, *, S=None, G=None,
           lam=None, tol: float = DEFAULT_TOL, dot="numpy", hutchpp: bool = True,
           gaussian: bool = False) -> Estimate:
    """log det Q by Algorithm 2 (each L-action by Algorithm 1), readings R2, R3,
    R5-R9, R14-R16."""
    Q = sp.csr_matrix(Q, dtype=np.float64)
    n = Q.shape[0]
    lam_lo, lam_hi = spectral_interval(Q, lam)
    gamma = math.sqrt(lam_lo * lam_hi)               # Proposition 2.1
    alpha = lam_lo                                   # R2
    shift = math.log(gamma / alpha)
    Qt = sp.csr_matrix((Q.data / gamma, Q.indices, Q.indptr), shape=Q.shape)
    s, r = _split(num_probes) if hutchpp else (0, num_probes)
    if S is not None:
        s = S.shape[1]
    if G is not None:
        r = G.shape[1]
    S, G = _probes(n, s, r, seed, S, G, gaussian)

    complex_logs: list = []

    def L_action(v):
        return iop_log_action(Qt, v, m, k, shift, tol, dot, complex_logs)

    flags = 0
    Y = (np.stack([L_action(S[:, i]) for i in range(s)], axis=1) if s
         else np.zeros((n, 0)))                                     # R8
    A = orth(Y)
    if A.shape[1] < s:
        flags |= FLAG_RANK_DEFICIENT
    per = []
    tr_sub = 0.0
    for i in range(A.shape[1]):
        qf = float(np.dot(A[:, i], L_action(A[:, i])))             # R7
        per.append(qf)
        tr_sub += qf
    Z = G - A @ (A.T @ G)
    zn2 = np.einsum("ij,ij->j", Z, Z)
    tr_res = 0.0
    for j in range(Z.shape[1]):
        if zn2[j] == 0.0:
            per.append(0.0)
            continue
        qf = float(np.dot(Z[:, j], L_action(Z[:, j])))
        per.append(qf / zn2[j])
        tr_res += qf
    tr_res /= r
    if complex_logs:
        flags |= FLAG_COMPLEX_LOG                    # R16
    logdet = n * math.log(alpha) + tr_sub + tr_res
    return Estimate(logdet, tr_sub, tr_res, math.log(alpha), math.log(gamma), s, r,
                    A.shape[1], np.array(per), zn2, flags)
