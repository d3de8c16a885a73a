"""Plants mistakes in the oracle (on the CPU) and checks that its pins catch each of them.

Each mutation is a one-line edit of the oracle's source (oracle/ttm.py), compiled into a
copy of the module. The pins are the ones of tests/test_oracle_ttm.py, restated compactly:
brute-force dense product, the discarded-weight error bound, single-swap optimality, the
Eq. eps rule cases, and the sin*cos closed form. The unmutated oracle passes all of them;
every mutation fails at least one.
"""

import importlib.util
import inspect

import numpy as np
import pytest

import ttgen
from oracle import tt
from oracle import ttm as ttm_orig

MUTATIONS = {
    # Fig. 1C / reading A2: the singular values go with the mover, not with V^T
    "absorb into the wrong carriage": [
        ("newY = (U[:, :k] * lam[:k]).reshape(Dl, d2, k)", "newY = U[:, :k].reshape(Dl, d2, k)"),
        ("newX = Vt[:k].reshape(k, d1, Dr)", "newX = (lam[:k, None] * Vt[:k]).reshape(k, d1, Dr)"),
    ],
    # reading A3: the gauge centre is moved by QR after every Contract
    "no QR gauge moves": [
        ("Pi[j], Pi[j + 1] = qr_move(Pi[j], Pi[j + 1])", "pass"),
        ("Pi[j], mover = qr_move(Pi[j], mover)", "pass"),
    ],
    # Fig. 1C: the two physical legs change places in a Swap
    "no leg permutation in the Swap": [
        ("theta = theta.transpose(0, 2, 1, 3)", "theta = theta"),
    ],
    # reading A1 / Eq. tensor: the reversed carriages have their bond legs exchanged
    "no bond-leg exchange in the reversal": [
        ("Mt = [m.transpose(2, 1, 0).copy() for m in Mc]", "Mt = [m.copy() for m in Mc]"),
    ],
    # reading A5: Eq. eps is a strict inequality
    "non-strict Eq. eps": [
        ("if tail[kk] < eps * total:", "if tail[kk] <= eps * total:"),
    ],
    # the discarded weight is the sum over the dropped values
    "off-by-one discarded weight": [
        ("return k, float(lam2[k:].sum())", "return k, float(lam2[k + 1:].sum())"),
    ],
}


def mutant(edits):
    src = inspect.getsource(ttm_orig)
    for old, new in edits:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    spec = importlib.util.spec_from_loader("oracle.ttm_mutant", loader=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__dict__["__package__"] = "oracle"
    exec(compile(src, "<mutant>", "exec"), mod.__dict__)
    return mod


# ---------------------------------------------------------------- the pins

def pin_dense(m):
    A = ttgen.rand_tt(8, 2, 4, 1000, canon="left")
    B = ttgen.rand_tt(8, 2, 3, 1100, canon="left")
    P = tt.dense(A) * tt.dense(B)
    O, _ = m.ttm(A, B)
    return np.linalg.norm(tt.dense(O) - P) <= 1e-12 * np.linalg.norm(P)


def pin_error_bound(m):
    A = ttgen.rand_tt(10, 2, 8, 11, canon="left")
    B = ttgen.rand_tt(10, 2, 8, 12, canon="left")
    P = tt.dense(A) * tt.dense(B)
    for eps, cap in ((1e-3, 0), (0.0, 6)):
        O, rep = m.ttm(A, B, eps=eps, chi_max=cap)
        if np.linalg.norm(tt.dense(O) - P) > rep["err_bound"] * (1 + 1e-9) + 1e-12 * np.linalg.norm(P):
            return False
    return True


def pin_single_swap(m):
    L = 6
    T = tt.left_canonical(ttgen.rand_tt(L, 2, 8, 91))
    newY, newX, lam, k, w = m.swap(T[L - 2], T[L - 1], eps=0.0, cap=2)
    before = tt.dense(T).reshape(2 ** (L - 2), 2, 2).transpose(0, 2, 1).reshape(-1)
    after = tt.dense(T[:L - 2] + [newY, newX])
    return abs(np.linalg.norm(before - after) - np.sqrt(w)) <= 1e-12 * np.linalg.norm(before)


def pin_eps_rule(m):
    lam = np.array([3.0, 2.0, 1.0, 0.5])
    tot = np.sum(lam ** 2)
    return (m.truncation_rank(lam, 0.25 / tot)[0] == 4 and m.truncation_rank(lam, 0.25 / tot + 1e-12)[0] == 3
            and m.truncation_rank(lam, 0.0, cap=2) == (2, 1.25))


def pin_closed_form(m):
    L = 10
    x = np.arange(2 ** L) / 2 ** L
    s = ttgen.qtt_trig(L, 2 * np.pi, 0.0, "sin")
    c = ttgen.qtt_trig(L, 2 * np.pi, 0.0, "cos")
    O, _ = m.ttm(s, c, eps=1e-24, chi_max=8)
    return max(tt.bonds_of(O)) <= 2 and np.abs(tt.dense(O) - 0.5 * np.sin(4 * np.pi * x)).max() <= 1e-12


PINS = [pin_dense, pin_error_bound, pin_single_swap, pin_eps_rule, pin_closed_form]


def run_pins(m):
    """Names of the pins that fail (an exception counts as a failure)."""
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
    failed = run_pins(mutant(MUTATIONS[name]))
    assert failed, "no pin catches: " + name
