"""The GEMM kernels through ttm_gemm: the float64 (DFMA) kernel and the tensor-core digit
product (TTM_PREC_BF16_SPLIT), against numpy's float64 matrix product.

Bounds: a float64 GEMM errs by at most about K u |A| |B| per entry (u = 2^-53), typically
sqrt(K) u. The digit product represents every scaled operand row / column to 2^-55 and sums
the digit products exactly, so its error stays within the same bound; the tests allow
4 K u |A||B| entrywise and 1e-14 relative in the Frobenius norm. Fewer digits (split_digits)
lose 7 bits each.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_19747_gb300 as p
    p.build()
    return p


def gemm(pkg, A, B, prec, **opts):
    h = pkg.Handle(0, **opts)
    try:
        C = pkg.ttm_gemm(h, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), prec=prec)
        torch.cuda.synchronize()
        return C.cpu().numpy()
    finally:
        h.close()


def check(A, B, C, entry_factor=4.0, rel=1e-14):
    ref = A @ B
    bound = entry_factor * A.shape[1] * U * (np.abs(A) @ np.abs(B)) + 1e-300
    assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)
    assert np.linalg.norm(C - ref) <= rel * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", ["fp64", "bf16_split"])
@pytest.mark.parametrize("M,N,K", [(128, 64, 32), (1, 1, 1), (200, 100, 70), (300, 257, 1000), (64, 130, 1500)])
def test_random(pkg, prec, M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    check(A, B, gemm(pkg, A, B, prec))


def test_split_graded_columns_keep_relative_accuracy(pkg):
    """Rows of A and columns of B spread over 30 decades: every row / column is scaled on
    its own, so each output entry keeps the float64 bound of its own row and column."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((256, 192)) * np.logspace(0, -30, 256)[:, None]
    B = rng.standard_normal((192, 128)) * np.logspace(5, -25, 128)[None, :]
    check(A, B, gemm(pkg, A, B, "bf16_split"))


def test_split_exact_on_small_integers(pkg):
    """Integer matrices whose products fit the digit range come out exactly."""
    rng = np.random.default_rng(6)
    A = rng.integers(-50, 50, (150, 300)).astype(np.float64)
    B = rng.integers(-50, 50, (300, 70)).astype(np.float64)
    C = gemm(pkg, A, B, "bf16_split")
    np.testing.assert_array_equal(C, A @ B)


@pytest.mark.parametrize("S", [3, 5])
def test_fewer_digits_lose_seven_bits_each(pkg, S):
    rng = np.random.default_rng(7)
    A = rng.standard_normal((128, 256))
    B = rng.standard_normal((256, 64))
    C = gemm(pkg, A, B, "bf16_split", split_digits=S)
    ref = A @ B
    err = np.linalg.norm(C - ref) / np.linalg.norm(ref)
    assert err <= 2.0 ** (-6 - 7 * (S - 1)) * 64
    assert err >= 2.0 ** (-6 - 7 * S) / 64     # the digits really are cut
