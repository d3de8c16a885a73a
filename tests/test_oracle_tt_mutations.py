"""Plants mistakes in oracle/tt.py (on the CPU) and checks that its pins catch each of them.

Each mutation is a one-line edit of the module's source compiled into a copy. References
come from the unmutated module (itself pinned in tests/test_oracle_tt.py), the quantities
under test from the mutant. The pins restate tests/test_oracle_tt.py: two-, three- and
four-layer environments against dense sums, the difference train, canonical forms, the
Kronecker cores of Eq. carriageXi, and dense gradients against central differences.
"""

import importlib.util
import inspect

import numpy as np
import pytest

import ttgen
from oracle import tt as tt_orig

MUTATIONS = {
    "two-layer environment transposed": [
        ("E = np.einsum('ab,asc,bsd->cd', E, Xk, Yk, optimize=True)",
         "E = np.einsum('ab,asc,bsd->dc', E, Xk, Yk, optimize=True)"),
    ],
    "three-layer environment joins W on another physical index": [
        ("En += np.tensordot(Wk[:, s, :], T2, axes=(0, 1))", "En += np.tensordot(Wk[:, (s + 1) % d, :], T2, axes=(0, 1))"),
    ],
    "difference train without the minus sign": [
        ("out.append(np.concatenate([Xk, -Yk], axis=2))", "out.append(np.concatenate([Xk, Yk], axis=2))"),
    ],
    "left-canonical sweep merges R transposed": [
        ("T[k + 1] = np.tensordot(R, T[k + 1], axes=(1, 0))", "T[k + 1] = np.tensordot(R.T, T[k + 1], axes=(1, 0))"),
    ],
    "Kronecker core pairs different physical indices": [
        ("P[:, s, :] = np.kron(Ka[:, s, :], Mb[:, s, :])", "P[:, s, :] = np.kron(Ka[:, s, :], Mb[:, (s + 1) % d, :])"),
    ],
    "gradient of <W, A o B> with the wrong factor": [
        ("gA = [_project_dense_gradient(w * b, A, k) for k in range(len(A))]",
         "gA = [_project_dense_gradient(w * a, A, k) for k in range(len(A))]"),
    ],
    "gradient of ||A o B - C||^2 without the factor 2": [
        ("gA = [_project_dense_gradient(2.0 * r * b, A, k) for k in range(len(A))]",
         "gA = [_project_dense_gradient(r * b, A, k) for k in range(len(A))]"),
    ],
    "gradient projection with exchanged bond legs": [
        ("return np.einsum('pa,psq,bq->asb', left, G, right, optimize=True)",
         "return np.einsum('pa,psq,bq->bsa', left, G, right, optimize=True)"),
    ],
    "squared distance with the cross term's sign flipped": [
        ("return ab2 - 2.0 * inner3(C, A, B) + inner(C, C)", "return ab2 + 2.0 * inner3(C, A, B) + inner(C, C)"),
    ],
}


def mutant(edits):
    src = inspect.getsource(tt_orig)
    for old, new in edits:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    spec = importlib.util.spec_from_loader("oracle.tt_mutant", loader=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__dict__["__package__"] = "oracle"
    exec(compile(src, "<mutant>", "exec"), mod.__dict__)
    return mod


A = ttgen.rand_tt(6, 2, 4, 41)
B = ttgen.rand_tt(6, 2, 3, 42)
W = ttgen.rand_tt(6, 2, 5, 43)
C = ttgen.rand_tt(6, 2, 2, 44)
a, b, w, c = (tt_orig.dense(X) for X in (A, B, W, C))


def close(x, ref, rel=1e-10):
    return abs(x - ref) <= rel * max(abs(ref), 1e-300)


def pin_inner(m):
    return close(m.inner(A, B), a @ b, 1e-12)


def pin_norm_and_diff(m):
    return close(m.norm(A), np.linalg.norm(a), 1e-12) and close(m.diff_norm(A, B), np.linalg.norm(a - b), 1e-12)


def pin_inner3(m):
    return close(m.inner3(W, A, B), float(np.sum(w * a * b)), 1e-12)


def pin_sqdist(m):
    return close(m.sqdist_via_environments(A, B, C), float(np.sum((a * b - c) ** 2)), 1e-10)


def pin_canonical(m):
    X = ttgen.rand_tt(6, 3, 5, 31)
    ref = tt_orig.dense(X)
    for T, side in ((m.left_canonical(X), "left"), (m.right_canonical(X), "right")):
        if np.abs(tt_orig.dense(T) - ref).max() > 1e-12 * np.abs(ref).max():
            return False
        for k in (range(5) if side == "left" else range(1, 6)):
            mm = T[k].reshape(-1, T[k].shape[2]) if side == "left" else T[k].reshape(T[k].shape[0], -1)
            g = mm.T @ mm if side == "left" else mm @ mm.T
            if np.abs(g - np.eye(g.shape[0])).max() > 1e-12:
                return False
    return True


def pin_kron(m):
    P = m.hadamard_kron(A, B)
    return np.abs(tt_orig.dense(P) - a * b).max() <= 1e-12 * np.abs(a * b).max()


def pin_gradients(m):
    L, d = 4, 3
    A_ = ttgen.rand_tt(L, d, 3, 51)
    B_ = ttgen.rand_tt(L, d, 2, 52)
    X_ = ttgen.rand_tt(L, d, 3, 53)
    x = tt_orig.dense(X_)
    for which in ("inner", "sqdist"):
        def f(Ap, Bp):
            r = tt_orig.dense(Ap) * tt_orig.dense(Bp)
            return float(np.sum(x * r)) if which == "inner" else float(np.sum((r - x) ** 2))
        val, gA, gB = m.grad_inner3_dense(X_, A_, B_) if which == "inner" else m.grad_sqdist_dense(A_, B_, X_)
        if not close(val, f(A_, B_), 1e-12):
            return False
        h = 1e-6
        for side, cores, grads in (("A", A_, gA), ("B", B_, gB)):
            for k in (0, L - 1):
                if grads[k].shape != cores[k].shape:
                    return False
                fd = np.zeros_like(cores[k])
                for idx in np.ndindex(cores[k].shape):
                    cp = [q.copy() for q in cores]
                    cm = [q.copy() for q in cores]
                    cp[k][idx] += h
                    cm[k][idx] -= h
                    fd[idx] = ((f(cp, B_) - f(cm, B_)) if side == "A" else (f(A_, cp) - f(A_, cm))) / (2 * h)
                if np.abs(grads[k] - fd).max() > 1e-6 * max(np.abs(grads[k]).max(), 1.0):
                    return False
    return True


PINS = [pin_inner, pin_norm_and_diff, pin_inner3, pin_sqdist, pin_canonical, pin_kron, pin_gradients]


def run_pins(m):
    failed = []
    for p in PINS:
        try:
            ok = p(m)
        except Exception:
            ok = False
        if not ok:
            failed.append(p.__name__)
    return failed


def test_unmutated_oracle_passes_every_pin():
    assert run_pins(mutant([])) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_each_planted_mistake_is_caught(name):
    assert run_pins(mutant(MUTATIONS[name])), "no pin catches: " + name
