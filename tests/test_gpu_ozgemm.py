"""FP64-accurate complex GEMM on the tensor cores (BF16 split products with
FP32 accumulation) against NumPy's FP64 product.

The scheme splits every row of op(A) and column of op(B) under its own power
of two into 6 slices of 7 bits, so its error is about 2^-42 of |A| |B|
(element-wise), independent of how the rows and columns are scaled; the
bounds asserted are 1e-11 |A| |B| element-wise and a relative Frobenius
error <= 2e-11 (the slicing error is 2^-43 of a row's largest entry, and a
product of random rows is about sqrt(K) smaller than |A| |B|).
Shapes cover ragged tails (M, N, K not multiples of the 128 x 64 tile or of
the 256-term exact chunk), both operand forms and a long inner dimension.
"""
import numpy as np
import pytest

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    return need_gpu()


def operands(m, n, k, seed, spread=6.0):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))) * 10.0 ** rng.uniform(-spread, 1, (m, 1))
    B = (rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))) * 10.0 ** rng.uniform(-spread, 1, (1, n))
    return A, B


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (7, 5, 3), (130, 70, 257), (300, 200, 600), (128, 64, 256),
                                   (513, 129, 1100), (64, 700, 2048)])
@pytest.mark.parametrize("opA,opB", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_oz_gemm_matches_fp64(M, m, n, k, opA, opB):
    import torch
    A, B = operands(m, n, k, seed=m * 7 + n + k)
    ref = A @ B
    At = torch.tensor(A.conj().T.copy() if opA else A, device="cuda")
    Bt = torch.tensor(B.conj().T.copy() if opB else B, device="cuda")
    C = M.gemm_ex(At, Bt, opA, opB, "fp64", engine=1).cpu().numpy()
    bound = np.abs(A) @ np.abs(B)
    assert np.all(np.abs(C - ref) <= 1e-11 * bound + 1e-300)
    assert np.linalg.norm(C - ref) <= 2e-11 * np.linalg.norm(ref)


def test_oz_gemm_zero_rows_and_columns(M):
    """Zero rows / columns (exponent 0 by convention) give exact zeros."""
    import torch
    A, B = operands(100, 90, 300, seed=3)
    A[5] = 0
    B[:, 7] = 0
    C = M.gemm_ex(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), 0, 0, "fp64", 1).cpu().numpy()
    assert np.all(C[5] == 0) and np.all(C[:, 7] == 0)
    assert np.linalg.norm(C - A @ B) <= 2e-11 * np.linalg.norm(A @ B)


def test_oz_gemm_more_accurate_than_fp32(M):
    """The point of the split: far below what an FP32 product can reach."""
    import torch
    A, B = operands(256, 128, 1024, seed=9, spread=0.0)
    ref = A @ B
    C = M.gemm_ex(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), 0, 0, "fp64", 1).cpu().numpy()
    C32 = (A.astype(np.complex64) @ B.astype(np.complex64)).astype(np.complex128)
    e64 = np.linalg.norm(C - ref) / np.linalg.norm(ref)
    e32 = np.linalg.norm(C32 - ref) / np.linalg.norm(ref)
    assert e64 < 2e-11 and e32 > 1e3 * e64
