"""The split-BF16 tcgen05 products (tensor cores, FP32 accumulation in
tensor memory) against FP64 products of the same operands."""
import numpy as np
import pytest

from tests.libutil import ensure_built

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hho():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ensure_built()


@pytest.mark.parametrize("K,N", [(16, 16), (32, 32), (64, 48), (48, 128)])
def test_split_bf16_gemm(hho, K, N):
    """Each operand is hi + lo in BF16 (16 significant bits); the dropped
    lo lo product and the FP32 accumulation leave an error of a few 2^-16
    of sum_k |a_k b_k|.  A distinct value in every entry catches any
    transposed or misplaced operand tile."""
    rng = np.random.default_rng(K * 1000 + N)
    A = rng.standard_normal((128, K)).astype(np.float32)
    B = rng.standard_normal((K, N)).astype(np.float32)
    D, status = hho.hho_tc_gemm_check(A, B)
    assert status == 0
    ref = A.astype(np.float64) @ B.astype(np.float64)
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    err = np.abs(D - ref) / scale
    print("K=%d N=%d: max |D - AB| / (|A||B|) = %.3e (2^-16 = %.3e)" % (K, N, err.max(), 2.0 ** -16))
    assert err.max() <= 4 * 2.0 ** -16
    # a single-term BF16 product would be far worse: the split is in effect
    assert err.max() <= 0.05 * np.abs(A.astype(np.float64)) .max() * 2.0 ** -8 * K or err.max() < 2.0 ** -14
