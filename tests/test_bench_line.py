"""bench.py's JSON line, assembled on the CPU from synthetic step reports.

The reports carry exactly the fields of the C report struct as the binding exposes them,
so a field renamed on one side and not the other fails here, not at the end of a GPU run.
"""

import json
import types

import numpy as np

import bench
from paper_2410_19747_gb300 import binding


def fake_report(**over):
    r = {f: 0 for f, _ in binding.c_report._fields_ if f != "bond_trace"}
    r.update(n_swaps=435, n_contracts=30, n_qr=435, max_bond=512, discarded_weight=2.8e-11,
             err_bound=1e-5, norm_out=1.1e-4, jacobi_sweeps_max=20, flops_counted=1.5e12,
             n_kernel_launches=12037, jacobi_launches=2 * 435, gemm_ms=9000.0, gemm_flops=9.0e12,
             gemm_launches=16 * 435, jacobi32_ms=12000.0, jacobi32_flops=3.0e16, qr_ms=3000.0)
    r.update(over)
    return r


def args(**over):
    a = dict(gpus=1, steps=1, warmup=3, impl="ours", chi=512, L=30, eps=1e-14, prec="fp64",
             no_cpu_baseline=False, e2e_steps=1, f32_passes=0, jacobi_kernel=0, batch=1, newton_steps=0,
             split_digits=0, time_budget=1500.0)
    a.update(over)
    return types.SimpleNamespace(**a)


def line_for(reps, t, **over):
    e2e = {"value": 1.0 / (t + 2.0), "unit": "products/s", "h2d_bytes_per_step": 10, "d2h_bytes_per_step": 5}
    clocks = {"sm_mhz": 1900.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 10}
    return bench.make_line(args(steps=len(reps), **over), reps, t, t, 1, e2e, clocks)


def test_contract_keys_and_values():
    line = line_for([fake_report()], 25.0)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    assert line["value"] == 1.0 / 25.0
    assert line["ms_per_step"] == 25000.0
    assert line["gpu_launches"] == 12037
    assert "workload" in line["config"]
    json.dumps(line)  # serialisable


def test_roofline_picks_the_dominant_kernel_family():
    roof = line_for([fake_report()], 25.0)["roofline"]
    # float32 Jacobi: 12 s of 25 s; GEMMs 9 s; QR 3 s
    assert roof["kernel"].startswith("jacobi_res_kernel<float>")
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert abs(roof["achieved"] - 3.0e16 / 12.0 / 1e12) < 1e-9
    assert abs(roof["frac"] - roof["achieved"] / bench.FP32_PEAK_TFLOPS) < 1e-12
    assert abs(roof["share_of_step"] - 12.0 / 25.0) < 1e-12
    other = roof["other_kernels"][0]
    assert other["kernel"].startswith("dgemm_kernel") and abs(other["achieved"] - 1.0) < 1e-12
    # GEMMs dominate: float64 pipe in fp64 mode, tensor pipe in the split mode
    roof = line_for([fake_report(gemm_ms=20000.0)], 35.0)["roofline"]
    assert roof["kernel"].startswith("dgemm_kernel") and roof["peak"] == bench.FP64_PEAK_TFLOPS
    roof = line_for([fake_report(gemm_ms=20000.0)], 35.0, prec="bf16_split")["roofline"]
    assert roof["bound"] == "tensor"
    assert abs(roof["achieved"] - 9.0e12 * 36 / 20.0 / 1e12) < 1e-6
    assert abs(roof["fp64_equivalent_tflops"] - 9.0e12 / 20.0 / 1e12) < 1e-9


def test_unprofiled_steps_give_no_rate():
    roof = line_for([fake_report(gemm_ms=0.0, jacobi32_ms=0.0, qr_ms=0.0)], 25.0)["roofline"]
    assert roof["achieved"] is None and roof["frac"] is None


def test_batched_steps_count_every_product():
    reps = [fake_report(), fake_report()]             # one launch-wide report per step
    line = bench.make_line(args(steps=2, batch=4), reps, 200.0, 200.0, 1,
                           {"value": None, "unit": "products/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                           {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0})
    assert line["value"] == 8 / 200.0
    assert line["config"]["batch"] == 4


def test_several_steps_sum():
    line = line_for([fake_report(), fake_report()], 50.0)
    assert line["value"] == 2.0 / 50.0
    assert line["gpu_launches"] == 2 * 12037
    assert line["steps"] == 2


def test_schedule_flops_match_the_oracles_realised_schedule():
    """bench.schedule_flops walks the schedule with the planner's upper bounds; on inputs
    where every cap binds (eps = 0, generic cores) these are the bonds the oracle realises,
    counted here by instrumenting the oracle's Swap, Contract and QR move."""
    import ttgen
    from oracle import ttm as ottm
    A = ttgen.rand_tt(9, 2, 12, 11)
    B = ttgen.rand_tt(9, 2, 10, 12)
    d, cap = 2, 16
    tot = [0.0]
    sw, co, qm = ottm.swap, ottm.contract, ottm.qr_move

    def swap(X, Y, eps=0.0, c=0):
        out = sw(X, Y, eps, c)
        tot[0] += bench.swap_model_flops(X.shape[0], X.shape[2], Y.shape[2], d, out[3])
        return out

    def contract(K, M):
        tot[0] += 2.0 * d * K.shape[0] * K.shape[2] * M.shape[2]
        return co(K, M)

    def qr_move(C, Cn):
        Q, R = qm(C, Cn)
        m, n, k, rr = d * C.shape[0], C.shape[2], Q.shape[2], Cn.shape[2]
        p, q = max(m, n), min(m, n)
        tot[0] += 2 * p * q * q - 2 / 3 * q ** 3 + 2 * m * k * k - 2 / 3 * k ** 3 + 2 * k * n * d * rr
        return Q, R

    try:
        ottm.swap, ottm.contract, ottm.qr_move = swap, contract, qr_move
        # the preparation's two QR sweeps are the oracle's left_canonical (not qr_move): count them apart
        from oracle import tt as ott
        lc = ott.left_canonical
        prep = [0.0]

        def left_canonical(T):
            bonds = [1] + [c.shape[2] for c in T]
            for k in range(len(T) - 1):
                m, n = d * bonds[k], bonds[k + 1]
                kk = min(m, n)
                p, q = max(m, n), min(m, n)
                prep[0] += (2 * p * q * q - 2 / 3 * q ** 3 + 2 * m * kk * kk - 2 / 3 * kk ** 3
                            + 2 * kk * n * d * bonds[k + 2])
                bonds[k + 1] = kk
            return lc(T)
        ott.left_canonical = left_canonical
        ottm.ttm(A, B, eps=0.0, chi_max=cap)
    finally:
        ottm.swap, ottm.contract, ottm.qr_move = sw, co, qm
        ott.left_canonical = lc
    got = bench.schedule_flops([1] + [c.shape[2] for c in A], [1] + [c.shape[2] for c in B], d, cap)
    assert abs(got - (tot[0] + prep[0])) <= 1e-9 * got


def test_accuracy_helpers_against_dense():
    """The bench's difference norm (QR sweep of the block-stacked difference) equals the dense
    2-norm of X - Y."""
    import ttgen
    from oracle import tt as ott
    X = ttgen.rand_tt(9, 2, 6, 81)
    Y = ttgen.rand_tt(9, 2, 5, 82)
    dx, dy = ott.dense(X), ott.dense(Y)
    assert abs(bench.tt_norm(X) - np.linalg.norm(dx)) <= 1e-12 * np.linalg.norm(dx)
    dd = np.linalg.norm(dx - dy)
    assert abs(bench.tt_norm(bench.stacked_difference(X, Y)) - dd) <= 1e-12 * dd
    assert bench.tt_norm(bench.stacked_difference(X, X)) <= 1e-13 * np.linalg.norm(dx)
