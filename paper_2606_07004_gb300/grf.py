"""Maximum-likelihood search for a Gaussian random field (Sec. 4, GRF study).

For each candidate theta the log-likelihood

    L(theta) = 1/2 log det Q(theta) - 1/2 x^T Q(theta) x - n/2 log(2 pi)

needs one log-determinant (OSA-IOP or OSLQ on the matrix-free gridded
Wendland operator Q(theta), support radius theta grid cells, plus a nugget)
and one quadratic form.  All candidates are submitted at once to a
continuous-batching server, so their Krylov steps share launches; the
quadratic forms run through logdet_quadform.  Every operation runs in the
CUDA library; this module only builds the tables and assembles L(theta).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import binding as B


@dataclass
class Sweep:
    theta: list
    logdet: list
    quad: list
    loglik: list
    theta_hat: float
    results: list = field(default_factory=list)


def wendland_c2(r):
    """Wendland's C^2 function for d <= 3: (1 - r)^4 (4 r + 1) on [0, 1), 0 beyond."""
    r = np.asarray(r, dtype=np.float64)
    return np.where(r < 1.0, (1.0 - r) ** 4 * (4.0 * r + 1.0), 0.0)


def wendland_table(theta: float, nugget: float) -> np.ndarray:
    """Quadrant table W[|dy|, |dx|] of the Wendland C^2 covariance with support
    radius theta grid cells, nugget added on the diagonal."""
    R = max(0, int(math.ceil(theta)) - 1)
    d = np.hypot(*np.meshgrid(np.arange(R + 1), np.arange(R + 1), indexing="ij"))
    W = wendland_c2(d / theta)
    W[0, 0] += nugget
    return W


def loglik_sweep(field_dev, nx: int, ny: int, thetas, *, nugget: float = 0.1,
                 method: int = B.METHOD_OSAIOP, num_probes: int = 21, krylov_steps: int = 20,
                 iop_window: int = 2, tol: float | None = 1e-6, precision: int = B.MIXED_FP32,
                 seed: int = 0, budget_bytes: int = 64 << 30, stream=None) -> Sweep:
    """L(theta) for every theta in `thetas`; field_dev is the observed field
    (nx * ny doubles on the device, row-major y * nx + x).  Defaults follow
    the paper's OSA-IOP run (m = 20, m_vec = 21, tol = 1e-6)."""
    n = nx * ny
    handles = [B.Handle.grid(nx, ny, wendland_table(float(t), nugget)) for t in thetas]
    try:
        with B.Server(budget_bytes, max_slots=len(handles), stream=stream) as srv:
            ids = [srv.submit(h, method, num_probes, krylov_steps, iop_window, seed=seed,
                              precision=precision, tol=tol) for h in handles]
            quads = [h.quadform(field_dev, stream=stream) for h in handles]
            res = [srv.wait(i) for i in ids]
    finally:
        for h in handles:
            h.close()
    logdets = [r.logdet for r in res]
    ll = [0.5 * ld - 0.5 * q - 0.5 * n * math.log(2.0 * math.pi) for ld, q in zip(logdets, quads)]
    best = int(np.argmax(ll))
    return Sweep(list(map(float, thetas)), logdets, quads, ll, float(thetas[best]), res)
