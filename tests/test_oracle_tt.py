"""Pins for oracle/tt.py against facts that do not come from the oracle itself:
closed forms, brute-force numpy, and finite differences."""

import numpy as np
import pytest

import ttgen
from oracle import tt


def test_bond_rule_formula_and_exactness():
    # Eq. bond with d=2: D_i = min(2^i, 2^(N-i), chi); chi_max = 2^floor(N/2) is exact (Sec. II).
    assert tt.bond_rule(7, 2, 0) == [1, 2, 4, 8, 8, 4, 2, 1]
    assert tt.bond_rule(8, 2, 5) == [1, 2, 4, 5, 5, 5, 4, 2, 1]
    rng = np.random.default_rng(7)
    for N in (5, 6, 7):
        x = rng.standard_normal(2 ** N)
        cores = ttgen.tt_svd(x, N, 2, chi=2 ** (N // 2))
        assert max(tt.bonds_of(cores)) <= 2 ** (N // 2)
        np.testing.assert_allclose(tt.dense(cores), x, rtol=0, atol=1e-12 * np.abs(x).max())


def test_dense_rank1_is_outer_product():
    rng = np.random.default_rng(1)
    vecs = [rng.standard_normal(3) for _ in range(5)]
    cores = [v.reshape(1, 3, 1) for v in vecs]
    ref = vecs[0]
    for v in vecs[1:]:
        ref = np.multiply.outer(ref, v)
    np.testing.assert_allclose(tt.dense(cores), ref.reshape(-1), rtol=1e-14, atol=0)


def test_dense_index_order_matches_matrix_product():
    # psi(s_1..s_L) = M^{s_1} ... M^{s_L} (Eq. TT), s_1 slowest.
    A = ttgen.rand_tt(4, 3, 3, 11)
    full = tt.dense(A).reshape(3, 3, 3, 3)
    for idx in [(0, 1, 2, 0), (2, 2, 1, 1), (1, 0, 0, 2)]:
        m = np.eye(1)
        for k, s in enumerate(idx):
            m = m @ A[k][:, s, :]
        assert abs(full[idx] - m[0, 0]) < 1e-12 * (1 + abs(m[0, 0]))


def test_qtt_generators_closed_forms():
    L = 12
    x = np.arange(2 ** L) / 2 ** L
    for om, ph in [(2 * np.pi, 0.0), (6 * np.pi, 0.3), (5.0, -1.0)]:
        np.testing.assert_allclose(tt.dense(ttgen.qtt_trig(L, om, ph, "cos")), np.cos(om * x + ph), atol=1e-13)
        np.testing.assert_allclose(tt.dense(ttgen.qtt_trig(L, om, ph, "sin")), np.sin(om * x + ph), atol=1e-13)
    np.testing.assert_allclose(tt.dense(ttgen.qtt_exp(L, 1.3)), np.exp(1.3 * x), rtol=1e-13)
    np.testing.assert_allclose(tt.dense(ttgen.qtt_linear(L, 0.5, -2.0)), 0.5 - 2.0 * x, atol=1e-13)


def test_kron_product_is_exact_hadamard():
    for d, ca, cb in [(2, 4, 3), (3, 3, 2)]:
        A = ttgen.rand_tt(5, d, ca, 21)
        B = ttgen.rand_tt(5, d, cb, 22)
        P = tt.hadamard_kron(A, B)
        ref = tt.dense(A) * tt.dense(B)
        np.testing.assert_allclose(tt.dense(P), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
        assert tt.bonds_of(P) == [a * b for a, b in zip(tt.bonds_of(A), tt.bonds_of(B))]


def test_canonical_forms():
    A = ttgen.rand_tt(6, 3, 5, 31)
    Lc = tt.left_canonical(A)
    Rc = tt.right_canonical(A)
    for k in range(5):
        c = Lc[k]
        m = c.reshape(-1, c.shape[2])
        np.testing.assert_allclose(m.T @ m, np.eye(m.shape[1]), atol=1e-12)
        c = Rc[k + 1]
        m = c.reshape(c.shape[0], -1)
        np.testing.assert_allclose(m @ m.T, np.eye(m.shape[0]), atol=1e-12)
    ref = tt.dense(A)
    np.testing.assert_allclose(tt.dense(Lc), ref, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(tt.dense(Rc), ref, atol=1e-12 * np.abs(ref).max())


def test_inner_norm_diffnorm_inner3_vs_dense():
    A = ttgen.rand_tt(6, 2, 4, 41)
    B = ttgen.rand_tt(6, 2, 3, 42)
    W = ttgen.rand_tt(6, 2, 5, 43)
    a, b, w = tt.dense(A), tt.dense(B), tt.dense(W)
    assert abs(tt.inner(A, B) - a @ b) <= 1e-12 * (np.abs(a) @ np.abs(b))
    assert abs(tt.norm(A) - np.linalg.norm(a)) <= 1e-12 * np.linalg.norm(a)
    assert abs(tt.diff_norm(A, B) - np.linalg.norm(a - b)) <= 1e-12 * np.linalg.norm(a - b)
    assert abs(tt.inner3(W, A, B) - np.sum(w * a * b)) <= 1e-12 * np.sum(np.abs(w * a * b))
    C = ttgen.rand_tt(6, 2, 2, 44)
    c = tt.dense(C)
    ref = np.sum((a * b - c) ** 2)
    assert abs(tt.sqdist_via_environments(A, B, C) - ref) <= 1e-10 * ref


def test_diff_norm_of_identical_tts_is_zero():
    A = ttgen.rand_tt(5, 2, 4, 45)
    assert tt.diff_norm(A, A) < 1e-13 * tt.norm(A)


@pytest.mark.parametrize("which", ["inner", "sqdist"])
def test_dense_gradients_match_central_differences(which):
    # dF/dcore by central differences (h = 1e-6, FP64) on every entry of a few cores.
    L, d = 5, 3
    A = ttgen.rand_tt(L, d, 3, 51)
    B = ttgen.rand_tt(L, d, 2, 52)
    X = ttgen.rand_tt(L, d, 3, 53)

    def f(A_, B_):
        a, b, x = tt.dense(A_), tt.dense(B_), tt.dense(X)
        if which == "inner":
            return float(np.sum(x * a * b))
        r = a * b - x
        return float(r @ r)

    if which == "inner":
        val, gA, gB = tt.grad_inner3_dense(X, A, B)
    else:
        val, gA, gB = tt.grad_sqdist_dense(A, B, X)
    assert abs(val - f(A, B)) <= 1e-12 * abs(val)
    h = 1e-6
    for side, cores, grads in [("A", A, gA), ("B", B, gB)]:
        for k in (0, 2, L - 1):
            g_fd = np.zeros_like(cores[k])
            for idx in np.ndindex(cores[k].shape):
                cp = [c.copy() for c in cores]
                cm = [c.copy() for c in cores]
                cp[k][idx] += h
                cm[k][idx] -= h
                if side == "A":
                    g_fd[idx] = (f(cp, B) - f(cm, B)) / (2 * h)
                else:
                    g_fd[idx] = (f(A, cp) - f(A, cm)) / (2 * h)
            scale = np.abs(grads[k]).max()
            assert np.abs(grads[k] - g_fd).max() <= 1e-6 * max(scale, 1.0)
