"""Pins for oracle/ttm.py (the paper's TTM on the CPU) against brute force, closed forms,
invariants the method fixes, and the worked example of Appendix A."""

import json
import os

import numpy as np
import pytest

import ttgen
from oracle import tt, ttm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- truncation rule (Eq. eps)

def test_truncation_rule_cases():
    lam = np.array([3.0, 2.0, 1.0, 0.5])
    tot = np.sum(lam ** 2)  # 14.25
    assert ttm.truncation_rank(lam, 0.0)[0] == 4                  # eps = 0 keeps everything
    assert ttm.truncation_rank(lam, 0.25 / tot + 1e-12)[0] == 3   # drops 0.5 (0.25 < eps*tot)
    assert ttm.truncation_rank(lam, 0.25 / tot)[0] == 4           # strict inequality
    assert ttm.truncation_rank(lam, 1.26 / tot)[0] == 2           # drops 1.0 and 0.5 (1.25)
    assert ttm.truncation_rank(lam, 0.999)[0] == 1                # never below one
    assert ttm.truncation_rank(lam, 0.0, cap=2) == (2, 1.25)      # cap and discarded weight
    assert ttm.truncation_rank(np.zeros(3), 0.1)[0] == 1          # zero tensor keeps one
    assert ttm.truncation_rank(np.array([1.0, 0.0, 0.0]), 0.0)[0] == 3  # eps=0 keeps zeros too


# ---------------------------------------------------------------- brute force and exact cases

@pytest.mark.parametrize("seed", [1000, 1001, 1002])
def test_untruncated_ttm_equals_dense_product(seed):
    # BJ config-1 shape: L=10, d=2, chi=8, left-canonical Gaussian cores.
    A = ttgen.rand_tt(10, 2, 8, seed, canon="left")
    B = ttgen.rand_tt(10, 2, 8, seed + 100, canon="left")
    P = tt.dense(A) * tt.dense(B)
    O, rep = ttm.ttm(A, B)
    assert np.linalg.norm(tt.dense(O) - P) <= 1e-12 * np.linalg.norm(P)
    # schedule of Sec. II.B: N contractions and N(N-1)/2 swaps
    assert rep["n_contracts"] == 10 and rep["n_swaps"] == 45
    assert rep["discarded_weight"] == 0.0


@pytest.mark.parametrize("d,L,ca,cb", [(3, 5, 4, 3), (4, 4, 5, 4)])
def test_untruncated_ttm_general_d(d, L, ca, cb):
    A = ttgen.rand_tt(L, d, ca, 7 + d)
    B = ttgen.rand_tt(L, d, cb, 8 + d)
    P = tt.dense(A) * tt.dense(B)
    O, rep = ttm.ttm(A, B)
    assert np.linalg.norm(tt.dense(O) - P) <= 1e-12 * np.linalg.norm(P)
    assert rep["n_swaps"] == L * (L - 1) // 2


def test_ttm_is_commutative_as_tensors():
    A = ttgen.rand_tt(8, 2, 6, 61)
    B = ttgen.rand_tt(8, 2, 5, 62)
    O1, _ = ttm.ttm(A, B)
    O2, _ = ttm.ttm(B, A)
    assert tt.diff_norm(O1, O2) <= 1e-12 * tt.norm(O1)


def test_rank_one_inputs_give_rank_one_product():
    rng = np.random.default_rng(3)
    L, d = 7, 3
    a = [rng.standard_normal(d) for _ in range(L)]
    b = [rng.standard_normal(d) for _ in range(L)]
    A = [v.reshape(1, d, 1) for v in a]
    B = [v.reshape(1, d, 1) for v in b]
    O, rep = ttm.ttm(A, B, eps=1e-20)
    assert tt.bonds_of(O) == [1] * (L + 1)
    assert rep["max_bond"] == 1
    ref = a[0] * b[0]
    for k in range(1, L):
        ref = np.multiply.outer(ref, a[k] * b[k])
    np.testing.assert_allclose(tt.dense(O), ref.reshape(-1), rtol=1e-12, atol=1e-14)


def test_constant_times_field_is_scaled_field():
    f = ttgen.rand_tt(8, 2, 6, 71)
    c = ttgen.constant_tt(8, 2, -2.5)
    O, _ = ttm.ttm(c, f, eps=1e-28)
    ref = -2.5 * tt.dense(f)
    assert np.linalg.norm(tt.dense(O) - ref) <= 1e-12 * np.linalg.norm(ref)
    assert max(tt.bonds_of(O)) <= max(tt.bonds_of(f))


def test_closed_form_qtt_products():
    L = 14
    x = np.arange(2 ** L) / 2 ** L
    # sin(2 pi x) cos(2 pi x) = sin(4 pi x) / 2 at rank 2 (chi_out = 2)
    s = ttgen.qtt_trig(L, 2 * np.pi, 0.0, "sin")
    c = ttgen.qtt_trig(L, 2 * np.pi, 0.0, "cos")
    O, rep = ttm.ttm(s, c, eps=1e-24, chi_max=8, chi_out=2)
    assert max(tt.bonds_of(O)) <= 2
    assert np.abs(tt.dense(O) - 0.5 * np.sin(4 * np.pi * x)).max() <= 1e-12
    # exp(a x) exp(b x) = exp((a+b) x) at rank 1
    O, rep = ttm.ttm(ttgen.qtt_exp(L, 0.7), ttgen.qtt_exp(L, -1.9), eps=1e-24)
    assert max(tt.bonds_of(O)) == 1
    np.testing.assert_allclose(tt.dense(O), np.exp(-1.2 * x), rtol=1e-12)
    # (x)(x) = x^2: ranks 2 x 2 -> 3
    lin = ttgen.qtt_linear(L, 0.0, 1.0)
    O, rep = ttm.ttm(lin, lin, eps=1e-26)
    assert max(tt.bonds_of(O)) == 3
    assert np.abs(tt.dense(O) - x ** 2).max() <= 1e-13


# ---------------------------------------------------------------- truncation error (Eq. eps + gauge)

@pytest.mark.parametrize("eps,cap", [(1e-6, 0), (1e-3, 0), (0.0, 6), (1e-10, 10)])
def test_truncation_error_within_discarded_weight(eps, cap):
    # In mixed canonical gauge a local truncation is a global one (statement next to Eq. eps):
    # the error of the product is bounded by sum_j sqrt(w_j). A wrong gauge breaks this.
    A = ttgen.rand_tt(10, 2, 8, 81, canon="left")
    B = ttgen.rand_tt(10, 2, 8, 82, canon="left")
    P = tt.dense(A) * tt.dense(B)
    O, rep = ttm.ttm(A, B, eps=eps, chi_max=cap)
    err = np.linalg.norm(tt.dense(O) - P)
    assert err <= rep["err_bound"] * (1 + 1e-9) + 1e-12 * np.linalg.norm(P)
    if cap:
        assert max(tt.bonds_of(O)) <= cap and rep["max_bond"] <= max(cap, 8)


def test_each_swap_truncation_is_globally_optimal_single_step():
    # One swap on a chain in mixed canonical gauge: the global error equals sqrt(w) exactly.
    L = 6
    T = tt.left_canonical(ttgen.rand_tt(L, 2, 8, 91))
    X, Y = T[L - 2], T[L - 1]           # centre on the right-most carriage of the pair
    newY, newX, lam, k, w = ttm.swap(X, Y, eps=0.0, cap=2)
    before = tt.dense(T).reshape(2 ** (L - 2), 2, 2)[:, :, :].transpose(0, 2, 1).reshape(-1)
    after = tt.dense(T[:L - 2] + [newY, newX])
    assert abs(np.linalg.norm(before - after) - np.sqrt(w)) <= 1e-12 * np.linalg.norm(before)


def test_scale_invariance():
    A = ttgen.rand_tt(9, 2, 8, 101, canon="left")
    B = ttgen.rand_tt(9, 2, 7, 102, canon="left")
    O1, r1 = ttm.ttm(A, B, eps=1e-8, chi_max=12)
    A2 = [c.copy() for c in A]
    A2[3] = A2[3] * 3.0
    O2, r2 = ttm.ttm(A2, B, eps=1e-8, chi_max=12)
    assert tt.bonds_of(O1) == tt.bonds_of(O2)
    O1s = [c.copy() for c in O1]
    O1s[0] = O1s[0] * 3.0
    assert tt.diff_norm(O1s, O2) <= 1e-10 * tt.norm(O2)


def test_bonds_respect_unfolding_bounds_and_caps():
    A = ttgen.rand_tt(10, 2, 8, 111, canon="left")
    B = ttgen.rand_tt(10, 2, 8, 112, canon="left")
    O, rep = ttm.ttm(A, B, chi_max=16, chi_out=12)
    D = tt.bonds_of(O)
    for i, Di in enumerate(D):
        assert Di <= min(2 ** i, 2 ** (10 - i), 12)
    assert rep["max_bond"] <= 16


# ---------------------------------------------------------------- conventional route (Sec. II.A)

def test_conventional_route_exact_and_bounded():
    A = ttgen.rand_tt(8, 2, 5, 121)
    B = ttgen.rand_tt(8, 2, 4, 122)
    P = tt.dense(A) * tt.dense(B)
    C, ws = ttm.conventional(A, B)
    assert np.linalg.norm(tt.dense(C) - P) <= 1e-12 * np.linalg.norm(P)
    C, ws = ttm.conventional(A, B, 0.0, 6)
    err = np.linalg.norm(tt.dense(C) - P)
    assert err <= np.sqrt(sum(ws)) * (1 + 1e-9)     # TT-SVD rounding bound (orthogonal truncations)
    # TTM with the same final cap is no worse than a small factor of the conventional route
    O, rep = ttm.ttm(A, B, chi_max=6, chi_out=6)
    assert np.linalg.norm(tt.dense(O) - P) <= 10 * err + 1e-12


# ---------------------------------------------------------------- Appendix A worked example

def _entropy(s):
    p = s ** 2 / np.sum(s ** 2)
    p = p[p > 1e-30]
    return float(-np.sum(p * np.log2(p)))


def test_appendix_a_swap_doubles_spectrum():
    g = json.load(open(os.path.join(GOLDEN, "appendix_a_toy.json")))
    M1 = np.array(g["carriage_1"]["values"])
    M2 = np.array(g["carriage_2"]["values"])
    two_bit = np.einsum('asb,btc->st', M1, M2)
    np.testing.assert_allclose(two_bit, np.array(g["two_bit_matrix"]), atol=1e-15)
    np.testing.assert_allclose(np.linalg.svd(two_bit, compute_uv=False), g["two_bit_singular_values"], atol=1e-15)
    N = 7
    rest = ttgen.rand_tt(N - 2, 2, 4, 131)          # arbitrary carriages 3..N (left bond 1)
    theta = [M1, M2] + rest
    full0 = tt.dense(theta).reshape((2,) * N)
    # move carriage 2 to the end with successive untruncated swaps
    chain = [c.copy() for c in theta]
    pos = 1
    while pos < N - 1:
        newY, newX, lam, k, w = ttm.swap(chain[pos], chain[pos + 1], eps=1e-24)
        chain[pos], chain[pos + 1] = newY, newX
        pos += 1
    full1 = tt.dense(chain).reshape((2,) * N)
    perm = [0] + list(range(2, N)) + [1]
    np.testing.assert_allclose(full1, full0.transpose(perm), atol=1e-13)
    # every cut after position p (p >= 2) in the new order: singular values (1/sqrt2, 1/sqrt2) x lam_init
    for p in range(2, N - 1):
        s_new = np.linalg.svd(full1.reshape(2 ** p, -1), compute_uv=False)
        s_init = np.linalg.svd(full0.reshape(2 ** (p + 1), -1), compute_uv=False)
        expect = np.sort(np.kron(np.array(g["two_bit_singular_values"]), s_init))[::-1]
        m = min(len(expect), len(s_new))
        np.testing.assert_allclose(s_new[:m], expect[:m], atol=1e-12)
        assert abs(_entropy(s_new) - _entropy(s_init) - g["entropy_increase_bits"]) < 1e-9
        assert tt.bonds_of(chain)[p] == 2 * int(np.sum(s_init > 1e-12))
