"""GPU parity of the TTM product (CUDA path through the C ABI) against the CPU oracle.

Tolerances: float64 untruncated products match the dense product to a relative
2-norm error of 1e-12; truncated products have an error against the exact
product within the oracle's own error plus 1e-10, and within the discarded-weight
bound sum_j sqrt(w_j)."""

import numpy as np
import pytest

import ttgen
from oracle import tt as ott
from oracle import ttm as ottm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_19747_gb300 as pkg
    pkg.build()
    hh = pkg.Handle(0)
    yield hh
    hh.close()


def dev(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cores]


def host(cores):
    return [c.cpu().numpy() for c in cores]


def run(h, A, B, **kw):
    import paper_2410_19747_gb300 as pkg
    out, rep = pkg.ttm_multiply(h, dev(A), dev(B), **kw)
    torch.cuda.synchronize()
    return host(out), rep


def relerr(O, P):
    return np.linalg.norm(ott.dense(O) - P) / np.linalg.norm(P)


@pytest.mark.parametrize("seed", [1000, 1001, 1002, 1003])
def test_config1_untruncated_matches_dense(h, seed):
    A = ttgen.rand_tt(10, 2, 8, seed, canon="left")
    B = ttgen.rand_tt(10, 2, 8, seed + 100, canon="left")
    P = ott.dense(A) * ott.dense(B)
    O, rep = run(h, A, B)
    assert relerr(O, P) <= 1e-12
    assert rep["n_swaps"] == 45 and rep["n_contracts"] == 10
    # eps = 0 keeps min(m, n) values; on wide Swap matrices the one-sided Jacobi leaves the
    # surplus columns at rounding level of the chain (norm ||A|| ||B||) instead of dropping
    # them structurally.
    chain2 = float(ott.dense(A) @ ott.dense(A)) * float(ott.dense(B) @ ott.dense(B))
    assert rep["discarded_weight"] <= 1e-26 * chain2
    Oo, ro = ottm.ttm(A, B)
    assert ott.bonds_of(O) == ott.bonds_of(Oo)


@pytest.mark.parametrize("seed", [1000, 1004])
def test_config1_truncated_within_oracle_error(h, seed):
    A = ttgen.rand_tt(10, 2, 8, seed, canon="left")
    B = ttgen.rand_tt(10, 2, 8, seed + 100, canon="left")
    P = ott.dense(A) * ott.dense(B)
    O, rep = run(h, A, B, chi_max=8, chi_out=8)
    Oo, ro = ottm.ttm(A, B, chi_max=8, chi_out=8)
    e_gpu, e_or = relerr(O, P), relerr(Oo, P)
    assert e_gpu <= e_or + 1e-10
    assert np.linalg.norm(ott.dense(O) - P) <= rep["err_bound"] * (1 + 1e-9)
    assert max(ott.bonds_of(O)) <= 8
    assert abs(rep["discarded_weight"] - ro["discarded_weight"]) <= 1e-9 * max(1.0, ro["discarded_weight"])


@pytest.mark.parametrize("d,L,ca,cb", [(3, 5, 4, 3), (4, 4, 5, 4), (4, 6, 7, 9), (8, 3, 8, 5)])
def test_general_d_untruncated(h, d, L, ca, cb):
    A = ttgen.rand_tt(L, d, ca, 7 + d + L)
    B = ttgen.rand_tt(L, d, cb, 8 + d + L)
    P = ott.dense(A) * ott.dense(B)
    O, rep = run(h, A, B)
    assert relerr(O, P) <= 1e-12
    assert rep["n_swaps"] == L * (L - 1) // 2


def test_edge_lengths(h):
    for L in (1, 2, 3):
        A = ttgen.rand_tt(L, 3, 4, 20 + L)
        B = ttgen.rand_tt(L, 3, 4, 30 + L)
        P = ott.dense(A) * ott.dense(B)
        O, rep = run(h, A, B)
        assert relerr(O, P) <= 1e-12


def test_closed_forms(h):
    L = 14
    x = np.arange(2 ** L) / 2 ** L
    s = ttgen.qtt_trig(L, 2 * np.pi, 0.0, "sin")
    c = ttgen.qtt_trig(L, 2 * np.pi, 0.0, "cos")
    # intermediate Swaps need more than rank 2; eps drops the exact zeros of the final rank-2 product
    O, rep = run(h, s, c, eps=1e-24, chi_max=8)
    assert max(ott.bonds_of(O)) <= 2
    assert np.abs(ott.dense(O) - 0.5 * np.sin(4 * np.pi * x)).max() <= 1e-12
    O, rep = run(h, ttgen.qtt_exp(L, 0.7), ttgen.qtt_exp(L, -1.9), eps=1e-24)
    assert max(ott.bonds_of(O)) == 1
    np.testing.assert_allclose(ott.dense(O), np.exp(-1.2 * x), rtol=1e-12)
    lin = ttgen.qtt_linear(L, 0.0, 1.0)
    O, rep = run(h, lin, lin, eps=1e-26)
    assert max(ott.bonds_of(O)) == 3
    # Rounding only: the sweep of Sec. II.B applies N(N-1)/2 = 91 Swap SVDs and 91 QR
    # gauge moves at N = 14, each an orthogonal factorisation that perturbs the product by
    # a few u (u = 2^-53) relative to max|x^2| = 1; 20u per factorisation gives 4e-13.
    assert np.abs(ott.dense(O) - x ** 2).max() <= 182 * 20 * 2.0 ** -53


def test_rank_one_and_constant(h):
    rng = np.random.default_rng(3)
    a = [rng.standard_normal(3).reshape(1, 3, 1) for _ in range(6)]
    b = [rng.standard_normal(3).reshape(1, 3, 1) for _ in range(6)]
    O, rep = run(h, a, b, eps=1e-20)
    assert ott.bonds_of(O) == [1] * 7
    assert relerr(O, ott.dense(a) * ott.dense(b)) <= 1e-13
    f = ttgen.rand_tt(8, 2, 6, 71)
    O, rep = run(h, ttgen.constant_tt(8, 2, -2.5), f, eps=1e-28)
    assert relerr(O, -2.5 * ott.dense(f)) <= 1e-12


def test_multi_tile_ragged_truncated(h):
    # bonds 70..100 span two 64-wide GEMM tiles with a ragged tail; eps-truncated and capped
    A = ttgen.rand_tt_spectral(14, 2, 70, 3100)
    B = ttgen.rand_tt_spectral(14, 2, 45, 3101)
    P = ott.dense(A) * ott.dense(B)
    for eps, cap in [(1e-10, 100), (1e-6, 0)]:
        O, rep = run(h, A, B, eps=eps, chi_max=cap, chi_out=cap)
        Oo, ro = ottm.ttm(A, B, eps=eps, chi_max=cap, chi_out=cap)
        e_gpu, e_or = relerr(O, P), relerr(Oo, P)
        assert e_gpu <= e_or + 1e-10, (e_gpu, e_or)
        assert np.linalg.norm(ott.dense(O) - P) <= rep["err_bound"] * (1 + 1e-9) + 1e-13 * np.linalg.norm(P)


def test_host_io_matches_device_io(h):
    import paper_2410_19747_gb300 as pkg
    A = ttgen.rand_tt(9, 2, 8, 501, canon="left")
    B = ttgen.rand_tt(9, 2, 8, 502, canon="left")
    Oh, rh = pkg.ttm_multiply(h, A, B, chi_max=12)   # numpy in, numpy out
    Od, rd = run(h, A, B, chi_max=12)
    assert ott.bonds_of(Oh) == ott.bonds_of(Od)
    for x, y in zip(Oh, Od):
        np.testing.assert_array_equal(x, y)


def test_batched_uneven_chi_equals_single(h):
    import paper_2410_19747_gb300 as pkg
    pairs = ttgen.pair_batch(5, 9, 2, 3, 16, 4000)
    res, reps = pkg.ttm_multiply_batched(h, [(dev(A), dev(B)) for A, B in pairs], chi_max=20)
    torch.cuda.synchronize()
    for (A, B), O, r in zip(pairs, res, reps):
        O1, r1 = run(h, A, B, chi_max=20)
        Oh = host(O)
        assert ott.bonds_of(Oh) == ott.bonds_of(O1)
        assert ott.diff_norm(Oh, O1) <= 1e-12 * ott.norm(O1)
        P = ott.dense(A) * ott.dense(B)
        assert np.linalg.norm(ott.dense(Oh) - P) <= r["err_bound"] * (1 + 1e-9) + 1e-12 * np.linalg.norm(P)


def test_batched_config4_shape(h):
    """A scaled-down config-4 batch: 8 random left-canonical pairs, L = 12, d = 2, bonds drawn
    from U{16..64}, multiplied in one ttm_multiply_batched call with chi_max = 48 in the mixed
    mode; every product equals its single call and stays within its error bound of the dense
    product."""
    import paper_2410_19747_gb300 as pkg
    pairs = ttgen.pair_batch(8, 12, 2, 16, 64, 4100)
    res, reps = pkg.ttm_multiply_batched(h, [(dev(A), dev(B)) for A, B in pairs], chi_max=48, eps=1e-14,
                                         prec="bf16_split")
    torch.cuda.synchronize()
    for (A, B), O, r in zip(pairs, res, reps):
        O1, r1 = run(h, A, B, chi_max=48, eps=1e-14, prec="bf16_split")
        Oh = host(O)
        assert ott.bonds_of(Oh) == ott.bonds_of(O1)
        assert ott.diff_norm(Oh, O1) <= 1e-9 * ott.norm(O1)
        P = ott.dense(A) * ott.dense(B)
        assert np.linalg.norm(ott.dense(Oh) - P) <= r["err_bound"] * (1 + 1e-9) + 1e-12 * np.linalg.norm(P)
