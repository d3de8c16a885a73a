"""bench.py's JSON line, assembled on the CPU from synthetic step reports.

The reports carry exactly the fields of the C report struct as the binding exposes them,
so a field renamed on one side and not the other fails here, not at the end of a GPU run.
"""

import json
import types

import bench
from paper_2410_19747_gb300 import binding


def fake_report(**over):
    r = {f: 0 for f, _ in binding.c_report._fields_ if f != "bond_trace"}
    r.update(n_swaps=435, n_contracts=30, n_qr=435, max_bond=512, discarded_weight=2.8e-11,
             err_bound=1e-5, norm_out=1.1e-4, jacobi_sweeps_max=30, flops_counted=2.0e12,
             n_kernel_launches=12037, jacobi_launches=4 * 435, jacobi_ms=17806.0,
             jacobi_flops=3.9e15, jacobi32_ms=70030.0, jacobi32_flops=4.0e16)
    r.update(over)
    return r


def args(**over):
    a = dict(gpus=1, steps=1, warmup=3, impl="ours", chi=512, L=30, eps=1e-14, prec="fp64",
             no_cpu_baseline=False, e2e_steps=1, f32_passes=0, f32_block=0, batch=1, polish_kd=0)
    a.update(over)
    return types.SimpleNamespace(**a)


def line_for(reps, t):
    e2e = {"value": 1.0 / (t + 2.0), "unit": "products/s", "h2d_bytes_per_step": 10, "d2h_bytes_per_step": 5}
    clocks = {"sm_mhz": 1900.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 10}
    return bench.make_line(args(steps=len(reps)), reps, t, t, 1, e2e, clocks)


def test_contract_keys_and_values():
    line = line_for([fake_report()], 118.0)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    assert line["value"] == 1.0 / 118.0
    assert line["ms_per_step"] == 118000.0
    assert line["gpu_launches"] == 12037
    assert "workload" in line["config"]
    json.dumps(line)  # serialisable


def test_roofline_picks_the_dominant_jacobi_kernel():
    roof = line_for([fake_report()], 118.0)["roofline"]
    # float32 passes: 70.0 s of 118 s; float64 polish: 17.8 s
    assert roof["kernel"].startswith("hestenes_kernel<float>")
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert abs(roof["achieved"] - 4.0e16 / 70.03 / 1e12) < 1e-9
    assert abs(roof["frac"] - roof["achieved"] / bench.FP32_PEAK_TFLOPS) < 1e-12
    assert abs(roof["share_of_step"] - 70.03 / 118.0) < 1e-12
    assert roof["launches"] == 3 * 435
    other = roof["other_kernels"][0]
    assert other["kernel"].startswith("hestenes_kernel<double>") and other["launches"] == 435
    # the other way round when the polish dominates
    roof = line_for([fake_report(jacobi_ms=90000.0, jacobi32_ms=10000.0)], 118.0)["roofline"]
    assert roof["kernel"].startswith("hestenes_kernel<double>")
    assert roof["peak"] == bench.FP64_PEAK_TFLOPS


def test_unprofiled_steps_give_no_rate():
    roof = line_for([fake_report(jacobi_ms=0.0, jacobi32_ms=0.0)], 118.0)["roofline"]
    assert roof["achieved"] is None and roof["frac"] is None


def test_batched_steps_count_every_product():
    reps = [fake_report(), fake_report()]             # one launch-wide report per step
    line = bench.make_line(args(steps=2, batch=4), reps, 200.0, 200.0, 1,
                           {"value": None, "unit": "products/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                           {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0})
    assert line["value"] == 8 / 200.0
    assert line["config"]["batch"] == 4
    assert line["roofline"]["launches"] == 2 * 3 * 435   # launches are shared by the batch


def test_several_steps_sum():
    line = line_for([fake_report(), fake_report()], 236.0)
    assert line["value"] == 2.0 / 236.0
    assert line["gpu_launches"] == 2 * 12037
    assert line["roofline"]["launches"] == 2 * 3 * 435
