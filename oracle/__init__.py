"""Plain FP64 CPU oracle for the OSLQ and OSA-IOP log-determinant estimators.

TEST INFRASTRUCTURE ONLY.  This package is the slow, literal reference that
the CUDA path is checked against.  Only the test suite, the smoke check and
the benchmark's CPU-baseline leg may import it; the library and its Python
binding never do, and they share no code with it (the two sides each
implement the probe generator from its published definition).

Contents
--------
``rademacher``  SplitMix64 counter-based Rademacher probes (the probe spec).
``estimators``  Algorithm 1 (Arnoldi-IOP-LOG), Algorithm 2 (OSA-IOP),
                Algorithm 3 (OSLQ), the Lanczos tridiagonalisation and the
                Gauss quadrature of Sec. 3.1, in NumPy/SciPy FP64.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, dense references, exactness cases and published generator
outputs; agreement with the paper's printed table values is unpinned because
the paper's test matrices are not available.
"""
from .rademacher import splitmix64_mix, rademacher_block, stream_key  # noqa: F401
from .estimators import (  # noqa: F401
    gershgorin_interval,
    spectral_interval,
    lanczos,
    gauss_quadrature_log,
    arnoldi_iop,
    iop_log_action,
    orth,
    oslq,
    osaiop,
)
