"""Benchmark of the GB300 TTM product (one JSON line on rank 0).

Workload (the metric's configuration): two random right-canonical tensor trains,
L = 30 sites, d = 2, bond chi = 512 with a 1/k profile inserted on every bond (the
realised Schmidt spectra decay faster), float64 cores; TTM with eps = 1e-14 and
chi_max = chi_out = 512. One step = one full
product (all N contractions, N(N-1)/2 swaps, all QR gauge moves) through the
C ABI. Inputs are resident in HBM for `value`; `e2e` repeats the step from
pinned host buffers with the copies inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--chi X]

Under torchrun (N > 1) every rank runs its own product (independent inputs, no
collective on the data path: weak scaling); rank 0 prints the line.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

T_START = time.monotonic()   # the --time-budget deadline counts from process start
ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TTM products/s + TFLOP/s at chi=512,d=2,L=30; mixed vs FP64 at rel err<=1e-7"
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12   # 2 DFMA/clk/SM x 152 SMs x 2.07 GHz = 1.259
FP32_PEAK_TFLOPS = 2 * 128 * 152 * 2.070e9 / 1e12  # 128 FFMA/clk/SM x 152 SMs x 2.07 GHz = 80.5
L2_BYTES = 129 * 2 ** 20
# DRAM bytes (read + write) per launch of a kernel, from the committed ncu captures (one launch
# each, named in the source); they describe the kernels as they are at the time of the capture.
MEASURED_TRAFFIC = {
    "jacobi_res_kernel<float>": (5.58e6, "profiles/jacobi_res_f32_chi512_L20.md: one full-size float32 pass "
                                         "(1024 x 1024, 70 ms); W and V stay in L2"),
    "oz_gemm_kernel": (7.29e6, "profiles/oz_gemm_gram_chi512_L20.md: one 1024^3 Gram"),
}
CPU_BASELINE_S = 40.0   # allowance for the CPU baseline leg in the --time-budget projection


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--chi", type=int, default=512)
    p.add_argument("--L", type=int, default=30)
    p.add_argument("--eps", type=float, default=1e-14)
    p.add_argument("--prec", default="bf16_split", choices=["fp64", "bf16_split"],
                   help="bf16_split (the mixed form, default): GEMMs as bf16 digit products on the tensor "
                        "cores; fp64: GEMMs on the float64 pipe")
    p.add_argument("--no-config1", action="store_true",
                   help="skip the small-bond side measurement (config 1: L=10, d=2, chi=8, float64)")
    p.add_argument("--no-accuracy", action="store_true",
                   help="skip the float64 product of the same inputs that the mixed result is compared with")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=1)
    p.add_argument("--f32-passes", type=int, default=0, help="float32 Jacobi passes (0: library default)")
    p.add_argument("--newton-steps", type=int, default=0, help="float64 Newton steps (0: library default)")
    p.add_argument("--split-digits", type=int, default=0, help="digits of bf16_split (0: library default)")
    p.add_argument("--batch", type=int, default=1,
                   help="independent products per step, multiplied in one ttm_multiply_batched call")
    p.add_argument("--jacobi-kernel", type=int, default=0, choices=[0, 1, 2, 3, 8, 16],
                   help="kernel of the float32 Jacobi passes (0: library default)")
    p.add_argument("--time-budget", type=float, default=1500.0,
                   help="seconds from process start by which the run should end: no timed step is "
                        "started that would end (with the e2e step and the CPU baseline) after it")
    return p.parse_args()


def workload(L, chi, seed):
    import ttgen
    A = ttgen.rand_tt_spectral(L, 2, chi, seed)
    B = ttgen.rand_tt_spectral(L, 2, chi, seed + 1)
    return A, B


def config(args):
    prec = getattr(args, "prec", "fp64")
    return {"workload": "config3: random right-canonical TT pair, L=%d, d=2, chi=%d, a 1/k profile on every "
                        "bond (realised Schmidt spectra steeper), float64 cores, eps=%g, chi_max=chi_out=%d"
                        % (args.L, args.chi, args.eps, args.chi),
            "L": args.L, "d": 2, "chi": args.chi, "eps": args.eps, "chi_out": args.chi,
            "precision_mode": prec, "batch": getattr(args, "batch", 1),
            "svd": "one-sided Jacobi, %d float32 passes (%s), then %d float64 Newton steps; GEMMs %s"
                   % (args.f32_passes or 3, {0: "default kernel", 1: "scalar kernel", 2: "two-column kernel",
                                             3: "resident-block kernel", 8: "Gram block 8",
                                             16: "Gram block 16"}[args.jacobi_kernel],
                      getattr(args, "newton_steps", 0) or 3,
                      "on the float64 pipe" if prec == "fp64" else
                      "as %d-digit bf16 products on the tensor cores" % (getattr(args, "split_digits", 0) or 8)),
            "l2": "flushed between timed steps (256 MiB write outside the timed events)"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def schedule_flops(bondsA, bondsB, d, chi_max):
    """Counted flops of one product (the model of Sec. II.B's schedule: Theta, SVD-equivalent
    Gram + U formation, Contract, Householder QR + R merge; Jacobi/Newton iterations
    excluded) with every bond at the upper bound the library's planner assigns it:
    min(d D_l, D_r) after a QR move, min(d D_l, d D_r, chi_max) after a Swap. When the caps
    bind (the metric's configuration) these are the realised bonds, and the count equals the
    report's flops_counted; the formulas are the library's."""
    L = len(bondsA) - 1
    bA, bB = list(bondsA), list(bondsB)
    fl = 0.0

    def qr(dl, dr, drr):
        m, n = d * dl, dr
        k = min(m, n)
        p, q = max(m, n), min(m, n)
        return k, 2 * p * q * q - 2 / 3 * q ** 3 + 2 * m * k * k - 2 / 3 * k ** 3 + 2 * k * n * d * drr

    for b in (bA, bB):                       # a1: both trains left-canonical
        for k in range(L - 1):
            nb, f = qr(b[k], b[k + 1], b[k + 2])
            fl += f
            b[k + 1] = nb
    mtL = [bB[L - j] for j in range(L)]      # Eq. tensor: B reversed, bond legs exchanged
    mtR = [bB[L - 1 - j] for j in range(L)]
    piL, piR = [0] * (L + 2), [0] * (L + 2)
    fl += 2 * d * bA[L - 1] * bA[L] * mtR[0]  # a2
    piL[L], piR[L] = bA[L - 1], mtR[0]
    for i in range(L - 1, 0, -1):
        mvR = mtR[L - i]
        for j in range(i + 1, L + 1):        # a3
            nxt = piR[j + 1] if j < L else mvR
            nb, f = qr(piL[j], piR[j], nxt)
            fl += f
            piR[j] = nb
            if j < L:
                piL[j + 1] = nb
        for j in range(L, i, -1):            # a4 + a5
            Dl, Dm, Dr = piL[j], piR[j], mvR
            nb = min(d * Dl, d * Dr)
            if chi_max > 0:
                nb = min(nb, chi_max)
            m, n = d * Dl, d * Dr
            fl += 2.0 * d * d * Dl * Dm * Dr + 2.0 * m * n * n + 2.0 * m * n * nb
            piL[j], piR[j], mvR = nb, mvR, nb
        fl += 2.0 * d * bA[i - 1] * bA[i] * mvR  # a6
        piL[i], piR[i] = bA[i - 1], mvR
    return fl


def swap_model_flops(Dl, Dm, Dr, d, k):
    m, n = d * Dl, d * Dr
    return 2.0 * d * d * Dl * Dm * Dr + 2.0 * m * n * n + 2.0 * m * n * k


def sample_carriages(args, A, B):
    """A full-size Swap of the benchmark workload: the carriage of A at the middle site made
    left-orthonormal (as the sweep holds it) and the middle carriage of the reversed B
    (bond legs exchanged, Eq. tensor) as the mover."""
    from oracle import tt as ott
    K = ott.left_canonical(A)
    Mc = ott.left_canonical(B)
    mid = len(A) // 2
    X = K[mid]
    Y = Mc[mid].transpose(2, 1, 0).copy()
    return X, Y


_SINGLE_CORE = r"""
import os, sys, time, json
sys.path.insert(0, %r)
import numpy as np
from oracle import ttm as ottm
d = np.load(%r)
X, Y = d["X"], d["Y"]
ottm.swap(X, Y, %r, %d)
t0 = time.perf_counter()
for _ in range(%d):
    ottm.swap(X, Y, %r, %d)
print(json.dumps({"dt": (time.perf_counter() - t0) / %d}))
"""


def time_oracle_swap(X, Y, eps, cap, n, threads):
    """Seconds per call of the oracle's Swap on (X, Y): in this process (all host threads of
    the BLAS) or, for threads == 1, in a child process started with one BLAS thread."""
    from oracle import ttm as ottm
    if threads != 1:
        ottm.swap(X, Y, eps, cap)
        t0 = time.perf_counter()
        for _ in range(n):
            ottm.swap(X, Y, eps, cap)
        return (time.perf_counter() - t0) / n
    import tempfile
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1")
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "xy.npz")
        np.savez(path, X=X, Y=Y)
        code = _SINGLE_CORE % (ROOT, path, eps, cap, n, eps, cap, n)
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        if out.returncode != 0:
            raise RuntimeError(out.stderr[-500:])
        return json.loads(out.stdout.strip().splitlines()[-1])["dt"]


def cpu_baseline(args, A, B, flops_product, n_multi=3, n_single=1):
    """The CPU float64 oracle timed on a bounded sample of the workload: full-size Swaps
    (oracle.ttm.swap: tensordot + LAPACK gesdd) on carriages of the benchmark inputs,
    extrapolated to one product by the counted flops of the product's schedule. Returns
    (products/s on all host threads, products/s on one core, description, seconds spent)."""
    t_start = time.perf_counter()
    X, Y = sample_carriages(args, A, B)
    f_swap = swap_model_flops(X.shape[0], X.shape[2], Y.shape[2], X.shape[1], args.chi)
    cores = os.cpu_count()
    dt_multi = time_oracle_swap(X, Y, args.eps, args.chi, n_multi, cores)
    try:
        dt_single = time_oracle_swap(X, Y, args.eps, args.chi, n_single, 1)
    except Exception:  # the single-core figure is context; the multi-thread one is the baseline
        dt_single = None
    per_product = dt_multi * flops_product / f_swap
    desc = ("%d full-size Swaps of the workload (oracle.ttm.swap on the left-orthonormal middle carriage "
            "of A and the middle carriage of the reversed B, %dx%dx%d and %dx%dx%d; numpy tensordot + "
            "LAPACK gesdd), %.3f s each on %d host threads%s; extrapolated to one product by counted flops "
            "(%.4g per product / %.4g per Swap)"
            % (n_multi, X.shape[0], X.shape[1], X.shape[2], Y.shape[0], Y.shape[1], Y.shape[2], dt_multi, cores,
               (", %.3f s on 1 core" % dt_single) if dt_single else "", flops_product, f_swap))
    single = (1.0 / (dt_single * flops_product / f_swap)) if dt_single else None
    return 1.0 / per_product, single, desc, time.perf_counter() - t_start


def run_reference(args, rank):
    """Reference arm: the CPU float64 oracle (the only other implementation of the paper
    here), on the bounded sample of cpu_baseline per step."""
    if rank != 0:
        return
    A, B = workload(args.L, args.chi, rank_seed(0))
    flops_product = schedule_flops([1] + [c.shape[2] for c in A], [1] + [c.shape[2] for c in B], 2, args.chi)
    for _ in range(args.warmup):
        cpu_baseline(args, A, B, flops_product, n_multi=1, n_single=0)
    vals, desc = [], ""
    spent = 0.0
    for _ in range(args.steps):
        v, _, desc, dt = cpu_baseline(args, A, B, flops_product, n_multi=1, n_single=0)
        vals.append(v)
        spent += dt
    value = float(np.mean(vals))
    _, single, _, _ = cpu_baseline(args, A, B, flops_product, n_multi=1, n_single=1)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "products/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
            "sample_s_per_step": spent / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args),
            "cpu_baseline": {"value": value, "unit": "products/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": desc, "value_1core": single},
            "e2e": {"value": value, "unit": "products/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def rank_seed(rank):
    """Seed of the rank's input pair: every rank multiplies its own independent pair (weak
    scaling; no collective on the data path)."""
    return 3000 + 10 * rank


def max_over_ranks(dist, x, device):
    """The largest x over all ranks (x itself without a process group)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    """The machine's measured peaks (generated MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"bf16_tflops": float(d["bf16_tflops"]), "bf16_tflops_sustained": float(d["bf16_tflops_sustained"]),
                "hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0, "source": "fallback"}


def kernel_roofline(args, reps, t_local):
    """Roofline object of the dominant kernel family of the timed steps (device time from CUDA
    events on the library's stream, summed over the launches of the family): the GEMMs
    (float64 pipe, or the tensor cores for bf16_split: digit products = S (S + 1) / 2 bf16
    GEMMs per algorithmic GEMM), the float32 one-sided Jacobi passes (flops counted on the
    device) or the Householder QR. The other families follow under "other_kernels"."""
    peaks = measured_peaks()
    S = getattr(args, "split_digits", 0) or 8
    tc = getattr(args, "prec", "fp64") == "bf16_split"
    kernels = []
    gemm_ms = sum(r["gemm_ms"] for r in reps)
    gemm_fl = sum(r["gemm_flops"] for r in reps)
    n_g = sum(r["gemm_launches"] for r in reps)
    if tc:
        ach = gemm_fl * S * (S + 1) / 2 / (gemm_ms / 1e3) / 1e12 if gemm_ms > 0 else None
        kernels.append({"bound": "tensor", "kernel": "oz_gemm_kernel (+ exponent and digit kernels): float64 "
                        "GEMMs as %d-digit bf16 tcgen05 products" % S, "achieved": ach,
                        "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                        "peak_source": "%s dense bf16, sustained (kernel timed inside a long step)" % peaks["source"],
                        "fp64_equivalent_tflops": (gemm_fl / (gemm_ms / 1e3) / 1e12) if gemm_ms > 0 else None,
                        "ms": gemm_ms, "launches": n_g})
    else:
        ach = gemm_fl / (gemm_ms / 1e3) / 1e12 if gemm_ms > 0 else None
        kernels.append({"bound": "alu", "kernel": "dgemm_kernel (float64 DFMA)", "achieved": ach,
                        "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "peak_source": "nominal float64 rate, 2 DFMA/clk/SM x 152 SMs x 2.07 GHz (a torch/cuBLAS "
                                       "DGEMM probe of this pool reached 1.10)",
                        "ms": gemm_ms, "launches": n_g})
    j_ms = sum(r["jacobi32_ms"] for r in reps)
    j_fl = sum(r["jacobi32_flops"] for r in reps)
    jk = getattr(args, "jacobi_kernel", 0)
    jname = {0: "jacobi_res_kernel<float> (resident-block one-sided Jacobi, float32)",
             1: "hestenes_kernel<float> (one-sided Jacobi, float32)",
             2: "jacobi4_kernel (two-column one-sided Jacobi, float32)",
             3: "jacobi_res_kernel<float> (resident-block one-sided Jacobi, float32)",
             8: "block_jacobi_kernel<8> (float32)", 16: "block_jacobi_kernel<16> (float32)"}[jk]
    kernels.append({"bound": "alu", "kernel": jname,
                    "achieved": (j_fl / (j_ms / 1e3) / 1e12) if j_ms > 0 else None, "peak": FP32_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "peak_source": "nominal float32 rate, 128 FFMA/clk/SM x 152 SMs x 2.07 GHz "
                                                      "(a torch SGEMM probe of this pool reached 69.8)",
                    "ms": j_ms, "launches": sum(r["jacobi_launches"] for r in reps)})
    kernels.append({"bound": "alu", "kernel": "jacobi_res_kernel<double> (float64 one-sided Jacobi of the "
                    "Newton fallback)", "achieved": None, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "ms": sum(r.get("jacobi64_ms", 0.0) for r in reps), "launches": None})
    kernels.append({"bound": "latency", "kernel": "householder_kernel (float64 QR of the gauge moves)",
                    "achieved": None, "peak": None, "unit": None, "ms": sum(r["qr_ms"] for r in reps),
                    "launches": None})
    for k in kernels:
        k["frac"] = (k["achieved"] / k["peak"]) if (k["achieved"] and k["peak"]) else None
        k["share_of_step"] = k["ms"] / 1e3 / t_local if t_local > 0 else None
        k["traffic"] = None
        for prefix, (nbytes, src) in MEASURED_TRAFFIC.items():
            if k["kernel"].startswith(prefix):
                k["traffic"] = nbytes
                k["traffic_source"] = src
    kernels.sort(key=lambda k: -(k["share_of_step"] or 0.0))
    roof = dict(kernels[0])
    roof["other_kernels"] = kernels[1:]
    return roof


def tt_norm(cores):
    """2-norm of a TT (host float64 arrays) by a left-orthogonalising QR sweep: the norm of the
    last core, without the cancellation of an inner-product sweep."""
    carry = None
    for k, c in enumerate(cores):
        c = c if carry is None else np.tensordot(carry, c, axes=(1, 0))
        a, d, b = c.shape
        if k == len(cores) - 1:
            return float(np.linalg.norm(c))
        q, carry = np.linalg.qr(c.reshape(a * d, b))
    return 0.0


def stacked_difference(X, Y):
    """Cores of the TT X - Y with block-stacked bonds (bond D_X + D_Y)."""
    L = len(X)
    out = []
    for k in range(L):
        x, y = X[k], Y[k]
        if L == 1:
            out.append(x - y)
        elif k == 0:
            out.append(np.concatenate([x, -y], axis=2))
        elif k == L - 1:
            out.append(np.concatenate([x, y], axis=0))
        else:
            c = np.zeros((x.shape[0] + y.shape[0], x.shape[1], x.shape[2] + y.shape[2]))
            c[:x.shape[0], :, :x.shape[2]] = x
            c[x.shape[0]:, :, x.shape[2]:] = y
            out.append(c)
    return out


def accuracy_vs_fp64(pkg, h, Ag, Bg, kw, out_mixed, rep_mixed, stream):
    """One float64 product (GEMMs on the float64 pipe) of the same inputs, timed on its own, and
    the relative 2-norm difference of the mixed result from it."""
    import torch
    kf = dict(kw, prec="fp64")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    of, rf = pkg.ttm_multiply(h, Ag, Bg, **kf)
    e1.record(stream)
    torch.cuda.synchronize()
    Om = [c.cpu().numpy() for c in out_mixed]
    Of = [c.cpu().numpy() for c in of]
    nf = tt_norm(Of)
    same = [c.shape for c in Om] == [c.shape for c in Of]
    diff = tt_norm(stacked_difference(Om, Of)) / nf if same else None
    return {"rel_err_vs_fp64": diff, "bound": 1e-7,
            "bonds_equal": same,
            "discarded_weight_rel_diff": abs(rep_mixed["discarded_weight"] - rf["discarded_weight"])
            / max(rf["discarded_weight"], 1e-300),
            "fp64_ms_per_product": e0.elapsed_time(e1), "fp64_status": rf["status"],
            "what": "||O_mixed - O_fp64||_2 / ||O_fp64||_2 of the last timed product against one float64 product "
                    "of the same inputs (host QR sweep of the block-stacked difference train)"}


def config1_throughput(pkg, h, dev, stream, warmup=5, steps=50):
    """Small-bond side measurement: products/s of config 1 (L = 10, d = 2, chi_A = chi_B =
    chi_out = 8, Gaussian cores left-canonicalised, float64 mode, eps = 0), inputs resident,
    CUDA events around `steps` back-to-back products after `warmup` untimed ones."""
    import torch
    import ttgen
    A = ttgen.rand_tt(10, 2, 8, 1000, canon="left")
    B = ttgen.rand_tt(10, 2, 8, 1100, canon="left")
    Ag = [torch.from_numpy(c).to(dev) for c in A]
    Bg = [torch.from_numpy(c).to(dev) for c in B]
    kw = dict(eps=0.0, chi_max=8, chi_out=8, prec="fp64")
    for _ in range(warmup):
        pkg.ttm_multiply(h, Ag, Bg, **kw)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        _, rep = pkg.ttm_multiply(h, Ag, Bg, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    out = {"workload": "config1: Gaussian TT pair, L=10, d=2, chi=8, left-canonicalised; float64, eps=0, "
                       "chi_max=chi_out=8", "products_per_s": 1e3 / ms, "ms_per_product": ms,
           "kernel_launches_per_product": rep["n_kernel_launches"], "steps": steps, "warmup": warmup,
           "note": "each call plans, allocates its arena and copies its report back; the time includes that host "
                   "work between the CUDA events"}
    try:  # the same with use_graph = 1: the first call captures the plan, the others replay it
        for _ in range(warmup):
            pkg.ttm_multiply(h, Ag, Bg, use_graph=1, **kw)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            pkg.ttm_multiply(h, Ag, Bg, use_graph=1, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        msg = e0.elapsed_time(e1) / steps
        out["graph"] = {"products_per_s": 1e3 / msg, "ms_per_product": msg}
    except Exception as ex:
        out["graph"] = {"error": repr(ex)}
    return out


def make_line(args, reps, t_local, t, world, e2e, clocks):
    """The bench JSON line (without cpu_baseline) from the reports of the timed steps, one
    report per step (launch-wide figures: a batched step shares its launches).
    t_local: this rank's summed step time; t: the max over ranks."""
    r0 = reps[-1]
    products = world * len(reps) * getattr(args, "batch", 1)
    flops = float(np.mean([r["flops_counted"] for r in reps]))
    return {
        "metric": METRIC, "value": products / t, "unit": "products/s", "n_gpus": world, "steps": len(reps),
        "warmup": args.warmup, "ms_per_step": 1e3 * t / len(reps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if getattr(args, "prec", "fp64") == "fp64" else
                 "mixed: f64 results, GEMMs as bf16 digit products (f32 accumulate), f32+f64 SVD",
        "data": "synthetic",
        "config": config(args),
        "tflops_counted": flops * products / t / 1e12,
        "roofline": kernel_roofline(args, reps, t_local),
        "e2e": e2e,
        "gpu_launches": int(sum(r["n_kernel_launches"] for r in reps)),
        "clocks": clocks,
        "report": {k: r0[k] for k in ("n_swaps", "n_contracts", "n_qr", "max_bond", "discarded_weight",
                                      "err_bound", "norm_out", "jacobi_sweeps_max", "newton_residual",
                                      "n_nonconverged", "status", "flops_counted")},
    }


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import torch
    import paper_2410_19747_gb300 as pkg
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    pkg.build()
    h = pkg.Handle(dev.index)
    host_pairs = [workload(args.L, args.chi, rank_seed(rank) + 100 * j) for j in range(args.batch)]
    pairs = [([torch.from_numpy(c).to(dev) for c in a], [torch.from_numpy(c).to(dev) for c in b])
             for a, b in host_pairs]
    Ag, Bg = pairs[0]
    kw = dict(eps=args.eps, chi_max=args.chi, chi_out=args.chi, prec=args.prec, f32_passes=args.f32_passes,
              jacobi_kernel=args.jacobi_kernel, newton_steps=args.newton_steps, split_digits=args.split_digits)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    last = {}

    def step(profile=0):
        """One step through the public call; returns the step's (launch-wide) report."""
        if args.batch == 1:
            out, rep = pkg.ttm_multiply(h, Ag, Bg, profile=profile, **kw)
            last["out"] = out
            return rep
        outs, reps_ = pkg.ttm_multiply_batched(h, pairs, profile=profile, **kw)
        last["out"] = outs[0]
        return reps_[0]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)

    reps, dts = [], []
    stopped = False
    with ClockSampler(dev.index) as clk:
        for q in range(args.steps):
            # no step is started that would end past the budget, counting the e2e steps and the
            # CPU baseline still to come (the ranks agree on the decision)
            if q > 0:
                mean = sum(dts) / len(dts)
                rest = mean * (1 + args.e2e_steps) + (0.0 if args.no_cpu_baseline else CPU_BASELINE_S + 20.0)
                if args.prec != "fp64" and not args.no_accuracy:
                    rest += 1.5 * mean + 10.0     # the float64 product and the host norm
                proj = max_over_ranks(dist, time.monotonic() - T_START + rest, dev)
                if proj > args.time_budget:
                    stopped = True
                    break
            flush.fill_(1.0)                       # L2 flush, outside the timed events
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rep = step(profile=1)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            dts.append(e0.elapsed_time(e1) / 1e3)
            reps.append(rep)
    torch.cuda.synchronize(dev)
    t_local = sum(dts)
    t = max_over_ranks(dist, t_local, dev)
    if dist:
        dist.barrier()

    # end to end through the public call from pinned host buffers
    e2e_t, h2d, d2h, e2e_err = 0.0, 0, 0, None
    try:
        hp = [([torch.from_numpy(c).pin_memory() for c in a], [torch.from_numpy(c).pin_memory() for c in b])
              for a, b in host_pairs]
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            if args.batch == 1:
                outs = [pkg.ttm_multiply(h, hp[0][0], hp[0][1], **kw)[0]]
            else:
                outs = pkg.ttm_multiply_batched(h, hp, **kw)[0]
            e2e_t += time.perf_counter() - t0
            h2d = sum(int(c.numel()) * 8 for a, b in hp for c in a + b)
            d2h = sum(int(c.numel()) * 8 for o in outs for c in o)
    except Exception as ex:  # the device-resident number above stays valid
        e2e_err = repr(ex)
    e2e_max = max_over_ranks(dist, e2e_t, dev)
    e2e_val = world * args.e2e_steps * args.batch / e2e_max if e2e_max > 0 else None

    # the mixed result against the float64 product of the same inputs (rank 0, untimed for value)
    accuracy = None
    if rank == 0 and args.prec != "fp64" and not args.no_accuracy and "out" in last:
        try:
            accuracy = accuracy_vs_fp64(pkg, h, Ag, Bg, kw, last["out"], reps[-1], stream)
        except Exception as ex:
            accuracy = {"error": repr(ex)}

    small = None
    if rank == 0 and not args.no_config1:
        try:
            small = config1_throughput(pkg, h, dev, stream)
        except Exception as ex:
            small = {"error": repr(ex)}

    if rank == 0:
        line = make_line(args, reps, t_local, t, world,
                         {"value": e2e_val, "unit": "products/s", "h2d_bytes_per_step": h2d,
                          "d2h_bytes_per_step": d2h, **({"error": e2e_err} if e2e_err else {})},
                         clk.summary())
        if accuracy is not None:
            line["accuracy"] = accuracy
        if small is not None:
            line["config1"] = small
        if stopped:
            line["steps_requested"] = args.steps
            line["stopped_early"] = ("the next step would have ended the run after --time-budget %.0f s "
                                     "(counted from process start)" % args.time_budget)
        flops = float(np.mean([r["flops_counted"] for r in reps]))
        if not args.no_cpu_baseline:
            A, B = host_pairs[0]
            v, v1, desc, spent = cpu_baseline(args, A, B, flops)
            line["cpu_baseline"] = {"value": v, "unit": "products/s", "cores": os.cpu_count(), "kind": "oracle",
                                    "sample": desc, "value_1core": v1, "sample_s": spent}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    h.close()


if __name__ == "__main__":
    main()
