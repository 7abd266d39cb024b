#!/usr/bin/env python
"""Benchmark of libkrr on GB300: Gaussian kernel MVP throughput and FGMRES
time-to-solution (the two halves of the headline metric).

One JSON line on rank 0.  A step is one full kernel product y = (K_hat +
gamma I) q through the C ABI on the 2^20-point unit-cube cloud (d = 3,
sigma 0.05, gamma 1e-3): point preparation (Morton sort, packing, block
metadata), the product kernel and its finalize.  `value` is whole-job
Gpairs/s (N^2 pairs per step per rank, all ranks, over the slowest rank's
device time).  Extra keys report the 16-column product, the FGMRES solves
(time to a 1e-6 relative residual, the plain float32 inner form next to the
reduced-precision inner form), the roofline of the product kernel, the
host-buffer end-to-end rate, the SM clocks seen during the timed region and
the FP64 oracle timed on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl libkrr|reference]
For N > 1 launch one process per GPU with torchrun; every rank solves its
own independent problem (seeded by rank) and ranks exchange only timings.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gaussian kernel MVP Gpairs/s; FGMRES time-to-1e-6 residual vs plain FP32 form"
# DRAM bytes (read + write) of one product-kernel launch on the 2^20-point
# workload, from one ncu capture (profiles/mvp_f32_kernel_cube1M_d3.md); valid
# only for the kernel source it was taken on.
TRAFFIC = {"source": "paper_1408_1237_gb300/csrc/mvp.cu", "sha1": "c6b59369cc94b9a6bbcad94ae2afbf5950649c4c",
           "bytes": 23.76e6 + 84.93e6}
MVP_N, MVP_D = 1 << 20, 3


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="libkrr", choices=["libkrr", "reference"])
    ap.add_argument("--solve-n", type=int, default=1 << 16,
                    help="points of the mixture-cloud FGMRES solve (0 skips it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args(argv)


# ------------------------------------------------------------ distributed ---
def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("KRR_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
    return rank, world, local


def max_over_ranks(value, world, device=None):
    """Largest value over all ranks (timing only; no data-path collective)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None and str(device).startswith("cuda"):
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def whole_job_rate(pairs_per_rank, world, seconds):
    """Aggregate Gpairs/s: all ranks' pairs over the slowest rank's time."""
    return pairs_per_rank * world / seconds / 1e9


# ----------------------------------------------------------------- clocks ---
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- reference ---
def cpu_oracle_rate(X, q, sigma, gamma, rows):
    """Oracle FP64 product on a row sample: returns (Gpairs/s, seconds, threads)."""
    import numpy as np
    import oracle
    oracle.build_oracle()
    X64 = X.astype(np.float64)
    q64 = q.astype(np.float64)
    t0 = time.perf_counter()
    oracle.mvp(X64, q64, sigma, gamma, rows=rows)
    dt = time.perf_counter() - t0
    return len(rows) * X.shape[0] / dt / 1e9, dt, oracle.num_threads()


def run_reference(args):
    rank, world, _ = dist_setup(args.gpus)
    if rank != 0:
        return 0
    from paper_1408_1237_gb300 import inputs
    p = inputs.mvp_problem(seed=0, N=MVP_N, d=MVP_D)
    rows_per_step = 1024
    for w in range(args.warmup):
        cpu_oracle_rate(p["X"], p["Q"], p["sigma"], p["gamma"],
                        inputs.sample_rows(MVP_N, rows_per_step, seed=100 + w))
    times, cores = [], 1
    for s in range(args.steps):
        rate, dt, cores = cpu_oracle_rate(p["X"], p["Q"], p["sigma"], p["gamma"],
                                          inputs.sample_rows(MVP_N, rows_per_step, seed=s))
        times.append(dt)
    pairs = rows_per_step * MVP_N
    value = pairs * len(times) / sum(times) / 1e9
    sample = f"{rows_per_step} seeded target rows x {MVP_N} sources per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gpairs/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"gaussian kernel product, N={MVP_N} uniform unit cube d=3, "
                               "sigma=0.05, gamma=1e-3, q~N(0,1), m=1 (FP64 oracle, row sample)"},
        "cpu_baseline": {"value": value, "unit": "Gpairs/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Gpairs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ libkrr ---
def run_libkrr(args):
    import numpy as np
    import torch

    rank, world, local = dist_setup(args.gpus)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1408_1237_gb300 import binding as K
    from paper_1408_1237_gb300 import inputs

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    # ---- headline product workload (seeded per rank: independent problems)
    p = inputs.mvp_problem(seed=rank, N=MVP_N, d=MVP_D)
    X = torch.from_numpy(p["X"]).to(dev)
    q = torch.from_numpy(p["Q"]).to(dev)
    y = torch.empty_like(q)
    sigma, gamma = p["sigma"], p["gamma"]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    for _ in range(max(args.warmup, 3)):
        K.krr_kernel_mvp(X, q, sigma, gamma, out=y)
    torch.cuda.synchronize(dev)

    ex2_rate, ffma_rate, ffma2_lanes = K.krr_measure_alu_peaks()
    fp32_lanes = max(ffma_rate, ffma2_lanes)
    # one MUFU.EX2 and d + 1 FP32 operations per pair (expanded form)
    peak_pairs = min(ex2_rate, fp32_lanes / (MVP_D + 1))

    barrier(world, dev)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    K.krr_profile_enable(True)
    launches0 = K.krr_profile_read()["launches"]
    K.krr_profile_enable(True)
    step_ms = []
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for s in range(args.steps):
        flush.zero_()  # untimed: evicts the inputs from L2 between steps
        evs[s][0].record(stream)
        K.krr_kernel_mvp(X, q, sigma, gamma, out=y)
        evs[s][1].record(stream)
    torch.cuda.synchronize(dev)
    prof = K.krr_profile_read()
    K.krr_profile_enable(False)
    barrier(world, dev)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_s = max_over_ranks(sum(step_ms) / 1e3, world, dev)
    pairs = float(MVP_N) * MVP_N
    value = whole_job_rate(pairs * args.steps, world, total_s)
    launches = prof["launches"] - launches0
    kern_ms = prof["product_ms"] / max(prof["product_launches"], 1)
    achieved = pairs / (kern_ms / 1e3) / 1e9

    # ---- 16 right-hand sides (one launch over all columns)
    Q16 = torch.from_numpy(inputs.mvp_problem(seed=rank + 7, N=MVP_N, d=MVP_D, m=16)["Q"].T.copy()).to(dev)
    Y16 = torch.empty_like(Q16)
    K.krr_kernel_mvp(X, Q16, sigma, gamma, out=Y16)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    K.krr_kernel_mvp(X, Q16, sigma, gamma, out=Y16)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    m16_ms = e0.elapsed_time(e1)

    # ---- end to end through the C ABI with pinned host buffers
    Xh = torch.from_numpy(p["X"]).pin_memory()
    qh = torch.from_numpy(p["Q"]).pin_memory()
    yh = torch.empty(MVP_N, dtype=torch.float32).pin_memory()
    K.krr_kernel_mvp(Xh, qh, sigma, gamma, out=yh)
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        K.krr_kernel_mvp(Xh, qh, sigma, gamma, out=yh)  # copies in, product, copy out, sync
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, dev)
    e2e_value = whole_job_rate(pairs, world, e2e_s)

    # ---- FGMRES time to a 1e-6 relative residual
    solve = {}
    sp = inputs.small_problem(seed=rank)
    solve["small_2000pt_2d"] = solve_once(K, torch, sp, dev, stream, "fp32")
    if args.solve_n > 0:
        mp = inputs.mixture_problem(seed=rank, N=args.solve_n)
        forms = {}
        for form in ("fp32", "bf16", "fp16"):
            try:
                forms[form] = solve_once(K, torch, mp, dev, stream, form)
            except K.KrrError as e:
                forms[form] = {"unavailable": str(e)}
        solve[f"mixture_{args.solve_n}pt_2d"] = forms

    # ---- FP64 oracle on the host cores (rank 0, one GPU only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nrows = 32768  # about 10 s of the oracle on 16 cores
        rows = inputs.sample_rows(MVP_N, nrows, seed=11)
        rate, dt, cores = cpu_oracle_rate(p["X"], p["Q"], sigma, gamma, rows)
        cpu = {"value": rate, "unit": "Gpairs/s", "cores": cores, "kind": "oracle",
               "sample": f"{nrows} seeded target rows x {MVP_N} sources ({dt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gpairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {
                "workload": f"gaussian kernel product y=(K_hat+gamma I)q, N={MVP_N} uniform "
                            "unit cube d=3, sigma=0.05, gamma=1e-3, q~N(0,1), m=1; step = "
                            "prep (Morton sort, pack) + product + finalize through the C ABI",
                "l2": "512 MB buffer written between timed steps (inputs are 16 MB)",
                "parallelism": f"{world} independent problems (one per GPU)",
            },
            "roofline": {
                "bound": "alu", "achieved": achieved, "peak": peak_pairs / 1e9,
                "unit": "Gpairs/s", "frac": achieved * 1e9 / peak_pairs, "traffic": traffic_bytes(),
                "kernel": "mvp_f32_kernel", "launch_ms": kern_ms,
                "peak_source": "measured on this GPU: min(MUFU.EX2 rate, FP32 lane rate/(d+1)) = "
                               f"min({ex2_rate / 1e12:.2f}e12, {fp32_lanes / 1e12:.2f}e12/{MVP_D + 1})",
            },
            "e2e": {"value": e2e_value, "unit": "Gpairs/s",
                    "h2d_bytes_per_step": MVP_N * (MVP_D + 1) * 4, "d2h_bytes_per_step": MVP_N * 4},
            "gpu_launches": launches,
            "clocks": clk,
            "mvp_m16": {"ms": m16_ms, "Gpair_rhs_per_s": pairs * 16 / (m16_ms / 1e3) / 1e9},
            "fgmres": solve,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def traffic_bytes():
    """ncu DRAM bytes per product launch, or None once the kernel changed."""
    import hashlib
    path = os.path.join(ROOT, TRAFFIC["source"])
    try:
        h = hashlib.sha1(open(path, "rb").read()).hexdigest()
    except OSError:
        return None
    return TRAFFIC["bytes"] if h == TRAFFIC["sha1"] else None


def solve_once(K, torch, p, dev, stream, inner_prec):
    """Time one FGMRES solve (prep included) with CUDA events; FP64-recheck
    is left to the tests.  Returns a report dict."""
    X = torch.from_numpy(p["X"]).to(dev)
    b = torch.from_numpy(p["b"]).to(dev)
    opts = K.default_opts(delta=p["delta"], inner_tol=p["inner_tol"], restart=p["restart"],
                          tol=p["tol"], inner_prec=inner_prec)
    warm = K.default_opts(restart=p["restart"], max_cycles=1, inner_maxit=1,
                          inner_prec=inner_prec)
    K.krr_fgmres_solve(X, b, p["sigma"], p["gamma"], opts=warm)  # allocates the workspace
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    x, info = K.krr_fgmres_solve(X, b, p["sigma"], p["gamma"], opts=opts)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    i = info[0]
    return {"time_to_solution_ms": e0.elapsed_time(e1), "relres_true": i["relres_true"],
            "outer": i["outer_iters"], "inner": i["inner_iters"], "cycles": i["cycles"],
            "status": K.status_string(i["status"]), "inner_prec": inner_prec,
            "N": int(p["X"].shape[0])}


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_libkrr(args)


if __name__ == "__main__":
    sys.exit(main())
