"""GPU checks that have not yet run on a GPU. They cover three paths: the final rounding to
chi_out < chi_max, the block float32 Jacobi (f32_block), and the kept/dropped-only float64
polish (polish_kept_dropped). There is also a full-size (chi = 512, L = 30) product check
against the oracle. pytest does not collect this module (no test_ prefix). Run it once on
its own (`python -m pytest tests/gpu_checks_pending.py -x -q`) and rename it to test_*.py
once it has passed.

Tolerances follow tests/test_gpu_ttm.py. The final rounding truncates bonds 1, 2, ... in the
oracle's order, so the products agree to rounding. The other two change only how the SVD
converges, so the results meet the same parity bounds as the default path.
"""

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


def run(h, A, B, **kw):
    import paper_2410_19747_gb300 as pkg
    out, rep = pkg.ttm_multiply(h, [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in A],
                                [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in B], **kw)
    torch.cuda.synchronize()
    return [c.cpu().numpy() for c in out], rep


def relerr(O, P):
    return np.linalg.norm(ott.dense(O) - P) / np.linalg.norm(P)


# ---------------------------------------------------------------- final rounding (a7)

@pytest.mark.parametrize("cap", [6, 3])
def test_final_rounding_matches_the_oracle(h, cap):
    A = ttgen.rand_tt_spectral(10, 2, 16, 11)
    B = ttgen.rand_tt_spectral(10, 2, 16, 12)
    O, rep = run(h, A, B, eps=1e-14, chi_max=32, chi_out=cap)
    Oo, ro = ottm.ttm(A, B, eps=1e-14, chi_max=32, chi_out=cap)
    assert ott.bonds_of(O) == ott.bonds_of(Oo)
    assert max(ott.bonds_of(O)) <= cap
    P = ott.dense(A) * ott.dense(B)
    assert np.linalg.norm(ott.dense(O) - ott.dense(Oo)) <= 1e-12 * np.linalg.norm(P)
    assert abs(rep["discarded_weight"] - ro["discarded_weight"]) <= 1e-9 * max(ro["discarded_weight"], 1e-300) + 1e-28
    assert np.linalg.norm(ott.dense(O) - P) <= rep["err_bound"] * (1 + 1e-9) + 1e-13 * np.linalg.norm(P)
    assert abs(rep["norm_out"] - np.linalg.norm(ott.dense(O))) <= 1e-12 * np.linalg.norm(ott.dense(O))
    assert rep["n_swaps"] == 45                       # the rounding SVDs are not Swaps


def test_final_rounding_closed_form(h):
    L = 14
    x = np.arange(2 ** L) / 2 ** L
    s = ttgen.qtt_trig(L, 2 * np.pi, 0.0, "sin")
    c = ttgen.qtt_trig(L, 2 * np.pi, 0.0, "cos")
    O, rep = run(h, s, c, eps=1e-24, chi_max=8, chi_out=2)
    assert max(ott.bonds_of(O)) <= 2
    assert np.abs(ott.dense(O) - 0.5 * np.sin(4 * np.pi * x)).max() <= 1e-12


def test_unbounded_swaps_with_output_cap(h):
    A = ttgen.rand_tt(8, 2, 6, 5, canon="left")
    B = ttgen.rand_tt(8, 2, 6, 6, canon="left")
    O, rep = run(h, A, B, eps=0.0, chi_max=0, chi_out=36)
    assert relerr(O, ott.dense(A) * ott.dense(B)) <= 1e-12      # a cap that binds nowhere


# ---------------------------------------------------------------- block float32 Jacobi

@pytest.mark.parametrize("fb", [8, 16])
def test_block_jacobi_untruncated_matches_dense(h, fb):
    for seed in (1000, 1001):
        A = ttgen.rand_tt(10, 2, 8, seed, canon="left")
        B = ttgen.rand_tt(10, 2, 8, seed + 100, canon="left")
        O, rep = run(h, A, B, f32_block=fb)
        assert relerr(O, ott.dense(A) * ott.dense(B)) <= 1e-12


@pytest.mark.parametrize("fb", [8, 16])
def test_block_jacobi_truncated_like_the_scalar_kernel(h, fb):
    A = ttgen.rand_tt_spectral(12, 2, 24, 3200)
    B = ttgen.rand_tt_spectral(12, 2, 20, 3201)
    P = ott.dense(A) * ott.dense(B)
    O0, r0 = run(h, A, B, eps=1e-10, chi_max=40, chi_out=40)
    O1, r1 = run(h, A, B, eps=1e-10, chi_max=40, chi_out=40, f32_block=fb)
    Oo, ro = ottm.ttm(A, B, eps=1e-10, chi_max=40, chi_out=40)
    e_or = np.linalg.norm(ott.dense(Oo) - P)
    assert np.linalg.norm(ott.dense(O1) - P) <= e_or + 1e-10
    assert abs(r1["discarded_weight"] - r0["discarded_weight"]) <= 1e-9 * max(1.0, r0["discarded_weight"])
    assert r1["jacobi32_flops"] > 0


# ---------------------------------------------------------------- kept/dropped polish

def test_kept_dropped_polish_where_the_cap_binds(h):
    A = ttgen.rand_tt_spectral(12, 2, 32, 41)
    B = ttgen.rand_tt_spectral(12, 2, 32, 42)
    P = ott.dense(A) * ott.dense(B)
    Of, rf = run(h, A, B, eps=1e-14, chi_max=16, chi_out=16)
    Ok, rk = run(h, A, B, eps=1e-14, chi_max=16, chi_out=16, polish_kept_dropped=1)
    Oo, ro = ottm.ttm(A, B, eps=1e-14, chi_max=16, chi_out=16)
    e_or = np.linalg.norm(ott.dense(Oo) - P)
    assert np.linalg.norm(ott.dense(Ok) - P) <= e_or + 1e-10 * np.linalg.norm(P)
    assert abs(rk["discarded_weight"] - rf["discarded_weight"]) <= 1e-8 * rf["discarded_weight"] + 1e-30
    assert rk["jacobi_flops"] < rf["jacobi_flops"]    # fewer float64 pair visits


def test_kept_dropped_polish_is_exact_when_nothing_is_cut(h):
    A = ttgen.rand_tt(10, 2, 8, 1000, canon="left")
    B = ttgen.rand_tt(10, 2, 8, 1100, canon="left")
    O, rep = run(h, A, B, polish_kept_dropped=1, chi_max=64)
    assert relerr(O, ott.dense(A) * ott.dense(B)) <= 1e-12


# ---------------------------------------------------------------- full size (config 3)

def test_full_size_config3_against_the_oracle(h):
    """chi = 512, L = 30, the benchmark's launch configuration, against the oracle's product
    on the same inputs (about 90 s on 16 host cores). Properties that hold at any size: the
    same bond trace, the same total discarded weight, and ||Omega_gpu - Omega_oracle|| small
    next to ||Omega||, measured with the two-layer environment on the GPU."""
    import paper_2410_19747_gb300 as pkg
    A = ttgen.rand_tt_spectral(30, 2, 512, 3000)
    B = ttgen.rand_tt_spectral(30, 2, 512, 3001)
    O, rep = run(h, A, B, eps=1e-14, chi_max=512, chi_out=512)
    Oo, ro = ottm.ttm(A, B, eps=1e-14, chi_max=512, chi_out=512)
    assert rep["n_swaps"] == 435 and rep["n_contracts"] == 30
    assert rep["bond_trace"] == ro["bond_trace"]
    assert abs(rep["discarded_weight"] - ro["discarded_weight"]) <= 1e-6 * ro["discarded_weight"]
    dev = lambda T: [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in T]
    g, o = dev(O), dev(Oo)
    gg, oo, go = pkg.ttm_inner(h, g, g), pkg.ttm_inner(h, o, o), pkg.ttm_inner(h, g, o)
    # the inner-product form of the distance has a floor near sqrt(u) * ||Omega||
    assert np.sqrt(max(gg + oo - 2 * go, 0.0) / oo) <= 1e-6
    assert abs(rep["norm_out"] - np.sqrt(oo)) <= 1e-9 * np.sqrt(oo)
