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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TTM products/s + TFLOP/s at chi=512,d=2,L=30; mixed vs FP64 at rel err<=1e-7"
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12   # 2 DFMA/clk/SM x 152 SMs x 2.07 GHz = 1.259
FP32_PEAK_TFLOPS = 2 * 128 * 152 * 2.070e9 / 1e12  # 128 FFMA/clk/SM x 152 SMs x 2.07 GHz = 80.5
L2_BYTES = 129 * 2 ** 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--chi", type=int, default=512)
    p.add_argument("--L", type=int, default=30)
    p.add_argument("--eps", type=float, default=1e-14)
    p.add_argument("--prec", default="fp64")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=1)
    p.add_argument("--f32-passes", type=int, default=0, help="float32 preconditioning passes (0: default)")
    p.add_argument("--batch", type=int, default=1,
                   help="independent products per step, multiplied in one ttm_multiply_batched call")
    p.add_argument("--polish-kd", type=int, default=0, choices=[0, 1],
                   help="1: float64 polish of the kept/dropped couplings only where the cap binds")
    p.add_argument("--f32-block", type=int, default=0, choices=[0, 8, 16],
                   help="block width of the float32 Jacobi (0: scalar kernel, the default)")
    return p.parse_args()


def workload(L, chi, seed):
    import ttgen
    A = ttgen.rand_tt_spectral(L, 2, chi, seed)
    B = ttgen.rand_tt_spectral(L, 2, chi, seed + 1)
    return A, B


def config(args):
    return {"workload": "config3: random right-canonical TT pair, L=%d, d=2, chi=%d, a 1/k profile on every "
                        "bond (realised Schmidt spectra steeper), float64 cores, eps=%g, chi_max=chi_out=%d"
                        % (args.L, args.chi, args.eps, args.chi),
            "L": args.L, "d": 2, "chi": args.chi, "eps": args.eps, "chi_out": args.chi,
            "precision_mode": args.prec, "batch": getattr(args, "batch", 1),
            "svd": "one-sided Jacobi: %d float32 passes (%s) + float64 polish (%s)"
                   % (args.f32_passes or 3, "block width %d" % args.f32_block if args.f32_block else "scalar",
                      "kept/dropped pairs where the cap binds" if getattr(args, "polish_kd", 0) else "all pairs"),
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


def cpu_baseline(args, flops_per_product, swap_flops_full, n_samples=2):
    """The oracle's Swap (numpy/LAPACK float64) on full-size carriages, extrapolated to one
    product by counted flops. Returns (products/s, seconds spent, description)."""
    from oracle import ttm as ottm
    rng = np.random.default_rng(7)
    chi = args.chi
    X = np.linalg.qr(rng.standard_normal((2 * chi, chi)))[0].reshape(chi, 2, chi)
    Y = rng.standard_normal((chi, 2, chi)) / chi
    t0 = time.perf_counter()
    for _ in range(n_samples):
        ottm.swap(X, Y, args.eps, chi)
    dt = (time.perf_counter() - t0) / n_samples
    per_product = dt * flops_per_product / swap_flops_full
    return 1.0 / per_product, dt * n_samples, (
        "%d full-size oracle Swaps (%dx2x%d carriages, numpy/LAPACK gesdd, %d host threads), "
        "%.2f s each, extrapolated to one product by counted flops (%.3g / %.3g)"
        % (n_samples, chi, chi, os.cpu_count(), dt, flops_per_product, swap_flops_full))


def swap_model_flops(chi):
    m = n = 2 * chi
    return 2.0 * 4 * chi ** 3 + 2.0 * m * n * n + 2.0 * m * n * chi


def model_flops(L, d, chi):
    """Counted flops of one product from the schedule of Sec. II.B with every bond at its
    upper bound min(d^i, d^(L-i), chi) (the same counting formulas the library applies
    to the realised bonds). Used only by the reference arm, which runs no GPU code."""
    ub = lambda i, n: min(chi, d ** min(i, n - i))
    fl = 0.0

    def qr(m, n, k, rr):
        p, q = max(m, n), min(m, n)
        return 2 * p * q * q - 2 / 3 * q ** 3 + 2 * m * k * k - 2 / 3 * k ** 3 + 2 * k * n * d * rr

    # preparation: two left-canonicalising QR sweeps
    for _ in range(2):
        for k in range(L - 1):
            Dl, Dr, Drr = ub(k, L), ub(k + 1, L), ub(k + 2, L)
            fl += qr(d * Dl, Dr, min(d * Dl, Dr), Drr)
    # sweep: iteration i moves the centre through Pi_{i+1}..Pi_N and swaps back
    for i in range(L - 1, 0, -1):
        for j in range(i + 1, L + 1):
            fl += qr(d * chi, chi, chi, chi)
        for j in range(L, i, -1):
            Dl = Dm = Dr = chi
            m = n = d * chi
            fl += 2.0 * d * d * Dl * Dm * Dr + 2.0 * m * n * n + 2.0 * m * n * chi
        fl += 2.0 * d * chi ** 3
    return fl


def run_reference(args, rank):
    """Reference arm: the CPU float64 oracle (the only implementation of the paper here)."""
    if rank != 0:
        return
    flops_product = model_flops(args.L, 2, args.chi)
    for _ in range(args.warmup):
        cpu_baseline(args, flops_product, swap_model_flops(args.chi), n_samples=1)
    vals, spent = [], 0.0
    desc = ""
    for _ in range(args.steps):
        v, s, desc = cpu_baseline(args, flops_product, swap_model_flops(args.chi), n_samples=1)
        vals.append(v)
        spent += s
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "products/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args),
            "cpu_baseline": {"value": value, "unit": "products/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": desc},
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


def jacobi_roofline(reps, t_local):
    """Roofline object of the dominant one-sided Jacobi kernel of the timed steps (device
    time from CUDA events on the library's stream, flops counted on the device), with the
    other Jacobi kernel attached under "other_kernels"."""
    kernels = []
    n_sw = sum(r["n_swaps"] for r in reps)
    for name, ms_key, fl_key, peak, src, n_l in (
            ("hestenes_kernel<double> (one-sided Jacobi polish, float64)", "jacobi_ms", "jacobi_flops",
             FP64_PEAK_TFLOPS, "nominal float64 rate: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz", n_sw),
            ("hestenes_kernel<float> (one-sided Jacobi preconditioning passes, float32)", "jacobi32_ms",
             "jacobi32_flops", FP32_PEAK_TFLOPS, "nominal float32 rate: 128 FFMA/clk/SM x 152 SMs x 2.07 GHz",
             sum(r["jacobi_launches"] for r in reps) - n_sw)):
        ms = sum(r[ms_key] for r in reps)
        fl = sum(r[fl_key] for r in reps)
        ach = (fl / (ms / 1e3) / 1e12) if ms > 0 else None
        kernels.append({"bound": "alu", "kernel": name, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                        "peak_source": src, "frac": (ach / peak) if ach else None, "traffic": None,
                        "share_of_step": ms / 1e3 / t_local if t_local > 0 else None,
                        "launches": n_l, "avg_launch_ms": ms / max(1, n_l)})
    kernels.sort(key=lambda k: -(k["share_of_step"] or 0.0))
    roof = dict(kernels[0])
    roof["other_kernels"] = kernels[1:]
    return roof


def make_line(args, reps, t_local, t, world, e2e, clocks):
    """The bench JSON line (without cpu_baseline) from the reports of the timed steps, one
    report per step (launch-wide figures: a batched step shares its launches).
    t_local: this rank's summed step time; t: the max over ranks."""
    r0 = reps[-1]
    products = world * args.steps * getattr(args, "batch", 1)
    flops = float(np.mean([r["flops_counted"] for r in reps]))
    return {
        "metric": METRIC, "value": products / t, "unit": "products/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config(args),
        "tflops_counted": flops * products / t / 1e12,
        "roofline": jacobi_roofline(reps, t_local),
        "e2e": e2e,
        "gpu_launches": int(sum(r["n_kernel_launches"] for r in reps)),
        "clocks": clocks,
        "report": {k: r0[k] for k in ("n_swaps", "n_contracts", "n_qr", "max_bond", "discarded_weight",
                                      "err_bound", "norm_out", "jacobi_sweeps_max")},
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
              f32_block=args.f32_block, polish_kept_dropped=args.polish_kd)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(profile=0):
        """One step through the public call; returns the step's (launch-wide) report."""
        if args.batch == 1:
            return pkg.ttm_multiply(h, Ag, Bg, profile=profile, **kw)[1]
        return pkg.ttm_multiply_batched(h, pairs, profile=profile, **kw)[1][0]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)

    reps, dts = [], []
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
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

    if rank == 0:
        line = make_line(args, reps, t_local, t, world,
                         {"value": e2e_val, "unit": "products/s", "h2d_bytes_per_step": h2d,
                          "d2h_bytes_per_step": d2h, **({"error": e2e_err} if e2e_err else {})},
                         clk.summary())
        flops = float(np.mean([r["flops_counted"] for r in reps]))
        if not args.no_cpu_baseline:
            v, spent, desc = cpu_baseline(args, flops, swap_model_flops(args.chi))
            line["cpu_baseline"] = {"value": v, "unit": "products/s", "cores": os.cpu_count(), "kind": "oracle",
                                    "sample": desc}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    h.close()


if __name__ == "__main__":
    main()
