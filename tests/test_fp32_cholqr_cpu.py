"""The precision argument behind the FP32 Hutch++ split of mixed-precision OSLQ,
checked on the CPU with NumPy: two rounds of Cholesky QR whose Gram matrix is
accurate (the GPU sums FP32 products with a compensated dot; here the products
of FP32 inputs are exact in FP64 and summed in FP64, at least as accurate), whose
Cholesky factor is FP64, and whose applies A = Y R^-1 run in FP32 with R^-1
rounded to FP32, leave A orthonormal to FP32 rounding for kappa(Y) up to 1e6
(the largest the column-drop rule |R_jj| > 1e-6 max |y| admits; measured
max |A^T A - I| ~1e-7 after two rounds, 4e-3 after one at kappa = 1e6), and
A spans the FP32 Y to FP32 rounding (relative residual <= 5e-7 measured).
This is an emulation of the arithmetic, not of the kernels; the kernels are
checked against the oracle on the GPU."""
import numpy as np
import pytest


def _gram(Y32):
    Y = Y32.astype(np.float64)
    return Y.T @ Y


def _round(Y32):
    C = _gram(Y32)
    R = np.linalg.cholesky(C).T                      # C = R^T R, upper R
    Rinv32 = np.linalg.inv(R).astype(np.float32)
    return (Y32 @ Rinv32).astype(np.float32)         # FP32 products and sums


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6])
@pytest.mark.parametrize("n,s", [(20000, 10), (5000, 40)])
def test_two_rounds_orthonormal_to_fp32_rounding(kappa, n, s):
    rng = np.random.default_rng(int(np.log10(kappa)) + s)
    Q, _ = np.linalg.qr(rng.standard_normal((n, s)))
    V, _ = np.linalg.qr(rng.standard_normal((s, s)))
    Y32 = (Q @ np.diag(np.logspace(0, -np.log10(kappa), s)) @ V.T).astype(np.float32)
    A1 = _round(Y32)
    A = _round(A1)
    A64 = A.astype(np.float64)
    orth = np.max(np.abs(A64.T @ A64 - np.eye(s)))
    assert orth < 1e-6
    # one round alone is not enough once kappa eps_32 is large
    if kappa >= 1e6:
        A1_64 = A1.astype(np.float64)
        assert np.max(np.abs(A1_64.T @ A1_64 - np.eye(s))) > 10 * orth
    # A spans the FP32 Y: the residual of Y after projection is FP32 rounding
    Y = Y32.astype(np.float64)
    res = Y - A64 @ (A64.T @ Y)
    assert np.linalg.norm(res) <= 2e-6 * np.linalg.norm(Y)
