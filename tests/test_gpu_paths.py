"""GPU parity of the paths beyond the default product: the final rounding to chi_out (a7,
reading A4), the block float32 Jacobi, the Newton refinement and its non-convergence
report, Swaps taller than one float32 register chunk (1024 rows), the config-2 turbulence
product and the metric's configuration (config 3: L = 30, d = 2, chi = 256 and 512)
against the oracle.

Tolerances follow tests/test_gpu_ttm.py: untruncated products match the dense product to
1e-12; truncated ones have an error against the exact product within the oracle's own
error plus 1e-10 (relative to ||A o B||) wherever the dense product fits in memory. At the
metric's sizes the exact product is out of reach; there the GPU and the oracle must agree
on the bond trace and the discarded weight, and the excess error eta of reading A10 (the
difference of the squared errors against A o B, evaluated exactly through the difference
and sum trains and the three-layer environment) must stay small.
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


def dev(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cores]


def run(h, A, B, **kw):
    import paper_2410_19747_gb300 as pkg
    out, rep = pkg.ttm_multiply(h, dev(A), dev(B), **kw)
    torch.cuda.synchronize()
    return [c.cpu().numpy() for c in out], rep


def relerr(O, P):
    return np.linalg.norm(ott.dense(O) - P) / np.linalg.norm(P)


def sum_tt(X, Y):
    """Block-stacked cores of X + Y (bond D_X + D_Y)."""
    L = len(X)
    out = []
    for k in range(L):
        a, b = X[k], Y[k]
        if L == 1:
            out.append(a + b)
        elif k == 0:
            out.append(np.concatenate([a, b], axis=2))
        elif k == L - 1:
            out.append(np.concatenate([a, b], axis=0))
        else:
            c = np.zeros((a.shape[0] + b.shape[0], a.shape[1], a.shape[2] + b.shape[2]))
            c[:a.shape[0], :, :a.shape[2]] = a
            c[a.shape[0]:, :, a.shape[2]:] = b
            out.append(c)
    return out


def excess_sq(h, Og, Oo, A, B):
    """||Og - A o B||^2 - ||Oo - A o B||^2 = <D, S> - 2 <D, A o B> with D = Og - Oo and
    S = Og + Oo, both as block-stacked trains: no difference of large numbers is formed."""
    import paper_2410_19747_gb300 as pkg
    D = ott.difference(Og, Oo)
    S = sum_tt(Og, Oo)
    dS = pkg.ttm_inner(h, dev(D), dev(S))
    dP = pkg.ttm_inner3(h, dev(D), dev(A), dev(B))
    return dS - 2.0 * dP


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
    # truncated results: compare errors against the exact product (reading A6), and the
    # two results only to well above the gap-limited non-uniqueness of the cut
    assert relerr(O, P) <= relerr(Oo, P) + 1e-10
    assert np.linalg.norm(ott.dense(O) - ott.dense(Oo)) <= 1e-10 * np.linalg.norm(P)
    assert abs(rep["discarded_weight"] - ro["discarded_weight"]) <= 1e-9 * ro["discarded_weight"] + 1e-28
    assert np.linalg.norm(ott.dense(O) - P) <= rep["err_bound"] * (1 + 1e-9) + 1e-13 * np.linalg.norm(P)
    assert abs(rep["norm_out"] - np.linalg.norm(ott.dense(O))) <= 1e-12 * np.linalg.norm(ott.dense(O))
    assert rep["n_swaps"] == 45                       # the rounding SVDs are not Swaps


def test_final_rounding_that_binds_nowhere_changes_nothing(h):
    """chi_out below chi_max but above every output bond: like the oracle, no bond is
    truncated, even with eps > 0 (the rounding applies only where a bond exceeds chi_out)."""
    A = ttgen.rand_tt_spectral(10, 2, 8, 21)
    B = ttgen.rand_tt_spectral(10, 2, 8, 22)
    O, rep = run(h, A, B, eps=1e-6, chi_max=12, chi_out=40)
    Oo, ro = ottm.ttm(A, B, eps=1e-6, chi_max=12, chi_out=40)
    assert ott.bonds_of(O) == ott.bonds_of(Oo)
    P = ott.dense(A) * ott.dense(B)
    assert relerr(O, P) <= relerr(Oo, P) + 1e-10
    assert np.linalg.norm(ott.dense(O) - ott.dense(Oo)) <= 1e-10 * np.linalg.norm(P)
    assert abs(rep["discarded_weight"] - ro["discarded_weight"]) <= 1e-9 * ro["discarded_weight"] + 1e-28


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


# ---------------------------------------------------------------- float32 Jacobi kernels
# 1: one column per tournament slot; 2: two columns per slot; 3: blocks of 8 columns resident
# in shared memory (the default up to 1024 rows); 8, 16: Gram-based blocks.

@pytest.mark.parametrize("fb", [1, 2, 3, 8, 16])
def test_block_jacobi_untruncated_matches_dense(h, fb):
    for seed in (1000, 1001):
        A = ttgen.rand_tt(10, 2, 8, seed, canon="left")
        B = ttgen.rand_tt(10, 2, 8, seed + 100, canon="left")
        O, rep = run(h, A, B, jacobi_kernel=fb)
        assert relerr(O, ott.dense(A) * ott.dense(B)) <= 1e-12


@pytest.mark.parametrize("fb", [1, 2, 3, 8, 16])
def test_block_jacobi_truncated_within_oracle_error(h, fb):
    A = ttgen.rand_tt_spectral(12, 2, 24, 3200)
    B = ttgen.rand_tt_spectral(12, 2, 20, 3201)
    P = ott.dense(A) * ott.dense(B)
    O1, r1 = run(h, A, B, eps=1e-10, chi_max=40, chi_out=40, jacobi_kernel=fb)
    Oo, ro = ottm.ttm(A, B, eps=1e-10, chi_max=40, chi_out=40)
    assert relerr(O1, P) <= relerr(Oo, P) + 1e-10
    assert abs(r1["discarded_weight"] - ro["discarded_weight"]) <= 1e-9 * max(1.0, ro["discarded_weight"])
    assert r1["jacobi32_flops"] > 0


# ---------------------------------------------------------------- Newton refinement

def test_newton_residual_reaches_rounding(h):
    A = ttgen.rand_tt_spectral(12, 2, 32, 41)
    B = ttgen.rand_tt_spectral(12, 2, 32, 42)
    O, rep = run(h, A, B, eps=1e-14, chi_max=16, chi_out=16)
    assert rep["status"] == 0 and rep["n_nonconverged"] == 0
    # the residual is the size of the last correction applied; convergence is quadratic, so a
    # last correction c leaves couplings of order c^2: 1e-9 leaves about 1e-18
    assert rep["newton_residual"] <= 1e-9


def test_non_convergence_is_reported(h):
    """max_sweeps = 1 (one sweep per float32 pass and for the float64 Jacobi of the fallback)
    and one Newton step cannot diagonalise these Swaps: the product is still returned, with
    TTM_WARN_NOT_CONVERGED in the report and the count of the SVDs."""
    A = ttgen.rand_tt_spectral(12, 2, 32, 41)
    B = ttgen.rand_tt_spectral(12, 2, 32, 42)
    O, rep = run(h, A, B, eps=1e-14, chi_max=16, chi_out=16, max_sweeps=1, newton_steps=1)
    assert rep["status"] == 1 and rep["status_name"] == "TTM_WARN_NOT_CONVERGED"
    assert rep["n_nonconverged"] > 0
    assert rep["n_fallback"] >= rep["n_nonconverged"]   # only the fallback's Jacobi counts


# ---------------------------------------------------------------- sizes

def test_swaps_taller_than_one_register_chunk(h):
    """d = 8, chi = 160: Swap matrices of 1280 rows (the float32 Jacobi keeps 1024 rows of a
    column pair in registers per pass), truncated by the cap, against the oracle."""
    A = ttgen.rand_tt_spectral(6, 8, 160, 3300)
    B = ttgen.rand_tt_spectral(6, 8, 150, 3301)
    P = ott.dense(A) * ott.dense(B)
    O, rep = run(h, A, B, eps=1e-12, chi_max=160, chi_out=160)
    Oo, ro = ottm.ttm(A, B, eps=1e-12, chi_max=160, chi_out=160)
    assert relerr(O, P) <= relerr(Oo, P) + 1e-10
    assert rep["n_nonconverged"] == 0


@pytest.mark.parametrize("chi_out", [64, 128])
def test_config2_turbulence_product(h, chi_out):
    """u * v of the 2D k^-5/3 turbulence fields (1024^2 grid, d = 4, TT-SVD to chi = 64)
    against the dense 1024^2 product."""
    u, v, _, _ = ttgen.turbulence_2d(L=10, chi=64, seed=2000)
    P = ott.dense(u) * ott.dense(v)
    O, rep = run(h, u, v, eps=1e-14, chi_max=chi_out, chi_out=chi_out)
    Oo, ro = ottm.ttm(u, v, eps=1e-14, chi_max=chi_out, chi_out=chi_out)
    assert relerr(O, P) <= relerr(Oo, P) + 1e-10
    assert np.linalg.norm(ott.dense(O) - P) <= rep["err_bound"] * (1 + 1e-9) + 1e-13 * np.linalg.norm(P)


def test_reduced_config3_within_oracle_error(h):
    """The metric's workload at L = 18, chi = 64 (dense product 2^18 entries)."""
    for seed in (3000, 3010):
        A = ttgen.rand_tt_spectral(18, 2, 64, seed)
        B = ttgen.rand_tt_spectral(18, 2, 64, seed + 1)
        P = ott.dense(A) * ott.dense(B)
        O, rep = run(h, A, B, eps=1e-14, chi_max=64, chi_out=64)
        Oo, ro = ottm.ttm(A, B, eps=1e-14, chi_max=64, chi_out=64)
        assert relerr(O, P) <= relerr(Oo, P) + 1e-10
        assert rep["bond_trace"] == ro["bond_trace"]


@pytest.mark.parametrize("chi", [256, 512])
def test_config3_against_the_oracle(h, chi):
    """L = 30, d = 2, eps = 1e-14, chi_max = chi_out = chi: the benchmark's configuration at
    chi = 512 (and 256), in the launch configuration bench.py times, against the oracle's
    product of the same inputs (tens of seconds on the host)."""
    A = ttgen.rand_tt_spectral(30, 2, chi, 3000)
    B = ttgen.rand_tt_spectral(30, 2, chi, 3001)
    O, rep = run(h, A, B, eps=1e-14, chi_max=chi, chi_out=chi)
    Oo, ro = ottm.ttm(A, B, eps=1e-14, chi_max=chi, chi_out=chi)
    assert rep["n_swaps"] == 435 and rep["n_contracts"] == 30
    assert rep["n_nonconverged"] == 0
    assert rep["bond_trace"] == ro["bond_trace"]
    assert abs(rep["discarded_weight"] - ro["discarded_weight"]) <= 1e-6 * ro["discarded_weight"]
    no2 = ott.inner(Oo, Oo)
    assert abs(rep["norm_out"] ** 2 - no2) <= 1e-9 * no2
    eta = np.sqrt(abs(excess_sq(h, O, Oo, A, B)) / no2)
    dist = ott.diff_norm(O, Oo) / np.sqrt(no2)
    print("chi %d: eta %.3e, distance to the oracle %.3e" % (chi, eta, dist))
    # measured on GB300: distance 2.5e-11 / 3.5e-11 and eta 5.0e-8 / 3.8e-8 at chi = 256 / 512
    assert dist <= 1e-8
    assert eta <= 1e-6


@pytest.mark.parametrize("chi", [128, 256])
def test_split_mode_against_fp64(h, chi):
    """The metric's gate for the mixed form: the tensor-core digit products (TTM_PREC_BF16_SPLIT)
    against the plain float64 GPU product on the config-3 workload, relative 2-norm difference
    ||O_split - O_fp64|| / ||O_fp64|| <= 1e-7, with the same bonds and discarded weight. The
    excess error eta (the difference of the squared errors against A o B, relative to the
    product's norm) is printed beside it: it grows like sqrt(difference x truncation error),
    about 1e-7 at chi = 128 where the truncation error is of the order of the product."""
    A = ttgen.rand_tt_spectral(30, 2, chi, 3000)
    B = ttgen.rand_tt_spectral(30, 2, chi, 3001)
    Of, rf = run(h, A, B, eps=1e-14, chi_max=chi, chi_out=chi)
    Om, rm = run(h, A, B, eps=1e-14, chi_max=chi, chi_out=chi, prec="bf16_split")
    assert rm["bond_trace"] == rf["bond_trace"]
    assert abs(rm["discarded_weight"] - rf["discarded_weight"]) <= 1e-6 * rf["discarded_weight"]
    nf2 = ott.inner(Of, Of)
    eta = np.sqrt(abs(excess_sq(h, Om, Of, A, B)) / nf2)
    dist = ott.diff_norm(Om, Of) / np.sqrt(nf2)
    print("chi %d: distance(split vs fp64) %.3e, eta %.3e" % (chi, dist, eta))
    assert dist <= 1e-7
