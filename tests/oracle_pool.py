"""Process pool for oracle work that splits into independent Krylov actions.

Full-size parity tests need tens of Algorithm-1 actions of the FP64 oracle on
a 2M-row matrix (seconds each); they are independent, so they run in worker
processes started with ``spawn`` (never forked from a process that holds a
CUDA context).  Each worker rebuilds the matrix from its seeded generator once
and imports neither torch nor the CUDA library.
"""
from __future__ import annotations

import math
import multiprocessing as mp
import os

_CACHE: dict = {}


def _matrix(spec):
    if spec not in _CACHE:
        import oracle as O
        import workloads as W
        kind, args = spec
        if kind != "laplacian_3d":
            raise ValueError(kind)
        Q = W.laplacian_3d(args[0], shift=args[1]).to_scipy()
        lo, hi = O.spectral_interval(Q)
        _CACHE.clear()
        _CACHE[spec] = (Q, lo, hi)
    return _CACHE[spec]


def _iop_action(job):
    """L v (Sec. 2.2) of one vector by Algorithm 1: job = (spec, v, m, k)."""
    import oracle as O
    spec, v, m, k = job
    Q, lo, hi = _matrix(spec)
    gamma = math.sqrt(lo * hi)
    return O.iop_log_action(Q / gamma, v, m, k, math.log(gamma / lo))


def _init(root):
    import sys
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    if root not in sys.path:
        sys.path.insert(0, root)


def make_pool(workers: int | None = None):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    n = workers or max(1, min(16, (os.cpu_count() or 1)))
    return mp.get_context("spawn").Pool(n, initializer=_init, initargs=(root,))


def iop_actions(pool, spec, vectors, m: int, k: int):
    """The oracle's L v for each column of ``vectors`` (n x c), in parallel."""
    jobs = [(spec, vectors[:, i].copy(), m, k) for i in range(vectors.shape[1])]
    return pool.map(_iop_action, jobs, chunksize=1)
