#!/usr/bin/env python
"""Benchmark of libkrr on GB300: Gaussian kernel MVP throughput and FGMRES
time-to-solution (the two halves of the headline metric).

One JSON line on rank 0.  A step is one full kernel product y = (K_hat +
gamma I) q through the C ABI on the 2^20-point unit-cube cloud (d = 3,
sigma 0.05, gamma 1e-3): point preparation (Morton sort, packing, block
metadata), the product kernel and its finalize.  `value` is whole-job
Gpairs/s (N^2 pairs per step per rank, all ranks, over the slowest rank's
device time).  Extra keys report the 16-column product, the roofline of the
product kernel, the host-buffer end-to-end rate, the SM clocks seen during
the timed region, the measured issue rates behind the design, and the FP64
oracle timed on the host cores.  On one GPU the solver forms follow, each
timed to a true relative residual of 1e-6: the batching workload at full
size (64 problems, mixed-precision and float32 batched calls against plain
float32 single-column solves), the precision-form mixture at full size
(262,144 points), every form compared on the same mixture at 65,536 points,
the log-marginal-likelihood gradient, and the high-d, Matern and autotuner
extras, in that order while the --budget-s wall clock lasts.

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
# DRAM bytes (read + write) of one product on the 2^20-point workload, from
# one ncu capture per path (dram__bytes_read.sum + dram__bytes_write.sum of
# every kernel of the product); valid only for the kernel sources they were
# taken on.
TRAFFIC = {"sources": {"paper_1408_1237_gb300/csrc/mvp.cu": "9775246cbc799cc4467e0840befecdb000cb45d1"},
           "bytes": 22374656 + 83717888}
# the same for the tensor-core exponent path (mvp_tcx_kernel + direct-form tail)
TRAFFIC_TCX = {"sources": {"paper_1408_1237_gb300/csrc/mvp.cu": "c97b0b9bbaaeb44ef0f54387704d2631a12ca666",
                           "paper_1408_1237_gb300/csrc/mvp_tc.cu": "56d5c2079577a7fb0c3bb0e0a57e1d21f79255e6"},
               "bytes": 22713600 + 92372480 + 17144576 + 0}
MVP_N, MVP_D = 1 << 20, 3


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="libkrr", choices=["libkrr", "reference"])
    ap.add_argument("--precision-n", type=int, default=1 << 18,
                    help="points of the full-size precision-form solve (the 16-component mixture; "
                         "plain FP32 inner products; 0 skips it)")
    ap.add_argument("--precision-cap", type=int, default=800,
                    help="inner CG steps per outer step of the precision-form solves")
    ap.add_argument("--solve-cap", type=int, default=400,
                    help="inner CG steps per outer step of the compared forms")
    ap.add_argument("--solve-n", type=int, default=1 << 16,
                    help="points of the mixture cloud on which every form is compared (plain FP32, "
                         "f16 and bf16 inner, 16-column blocks; 0 skips it)")
    ap.add_argument("--plain-cols", type=int, default=2,
                    help="right-hand sides solved one at a time for the per-RHS plain FP32 time")
    ap.add_argument("--batch-probs", type=int, default=64,
                    help="problems of the batching form (0 skips it)")
    ap.add_argument("--batch-nmax", type=int, default=65536,
                    help="largest problem of the batching form")
    ap.add_argument("--batch-plain", type=int, default=8,
                    help="seeded sample of problems solved one right-hand side at a time for the "
                         "plain FP32 per-RHS time of the batching form")
    ap.add_argument("--batch-fp16", action="store_true",
                    help="also time the batching form with f16 inner products")
    ap.add_argument("--grad-n", type=int, default=1 << 16,
                    help="points of the log-marginal-likelihood gradient (0 skips it)")
    ap.add_argument("--budget-s", type=float, default=660.0,
                    help="wall-clock seconds after which the remaining extra forms are skipped")
    ap.add_argument("--no-matern", dest="matern", action="store_false",
                    help="skip the Matern-kernel product and solves")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip the autotuned-plan comparison")
    ap.add_argument("--no-highd", dest="highd", action="store_false",
                    help="skip the high-dimensional product comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    a = ap.parse_args(argv)
    a.batch_forms = [("batched_fp32_inner", "fp32")] + ([("batched_fp16_inner", "fp16")] if a.batch_fp16 else [])
    return a


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
def cpu_oracle_rate(X, q, sigma, gamma, rows, with_values=False):
    """Oracle FP64 product on a row sample: returns (Gpairs/s, seconds,
    threads) and, with_values, the sampled rows' values."""
    import numpy as np
    import oracle
    oracle.build_oracle()
    X64 = X.astype(np.float64)
    q64 = q.astype(np.float64)
    t0 = time.perf_counter()
    y = oracle.mvp(X64, q64, sigma, gamma, rows=rows)
    dt = time.perf_counter() - t0
    out = (len(rows) * X.shape[0] / dt / 1e9, dt, oracle.num_threads())
    return out + (y,) if with_values else out


def cpu_oracle_solves(p):
    """The FP64 oracle's own solves of the 2000-point problem, timed on the
    host cores beside the GPU's: dense K, the Cholesky direct solve, and the
    paper's FGMRES with truncated-CG inner solves (same restart, delta and
    tolerances as the GPU run), both on dense NumPy products."""
    import numpy as np
    import oracle
    f32 = lambda v: float(np.float32(v))
    X, b = p["X"].astype(np.float64), p["b"].astype(np.float64)
    sigma, gamma, delta = f32(p["sigma"]), f32(p["gamma"]), f32(p["delta"])
    t0 = time.perf_counter()
    Kmat = oracle.regularised_matrix(X, sigma, gamma)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    x_direct = oracle.direct_solve(Kmat, b)
    t_direct = time.perf_counter() - t0
    Mmat = Kmat + delta * np.eye(len(b))
    t0 = time.perf_counter()
    res = oracle.krr_fgmres(lambda v: Kmat @ v, lambda v: Mmat @ v, b, restart=p["restart"],
                            tol=p["tol"], inner_tol=p["inner_tol"])
    t_fgmres = time.perf_counter() - t0
    rel = lambda x: float(np.linalg.norm(b - Kmat @ x) / np.linalg.norm(b))
    return {"N": int(len(b)), "dense_K_ms": t_build * 1e3,
            "cholesky_ms": t_direct * 1e3, "cholesky_relres": rel(x_direct),
            "fgmres_ms": t_fgmres * 1e3, "fgmres_relres": rel(res.x),
            "fgmres_outer": int(res.outer_iters), "fgmres_inner": int(res.inner_iters),
            "threads": "NumPy/SciPy BLAS defaults"}


def precision_errors(K, X, q, y32, sigma, gamma, p, rows, ref):
    """Max error per element of the float32, f16 and bf16 products (the
    last two: the inner-product precisions of the solver) against the FP64
    oracle on sampled rows, each scaled by the row's summation scale
    sum_j |q_j| K_hat_ij + gamma |q_i| (the oracle on the rows' |q|)."""
    import numpy as np
    import oracle
    f32 = lambda v: float(np.float32(v))
    scale = oracle.mvp(p["X"].astype(np.float64), np.abs(p["Q"].astype(np.float64)), f32(sigma), f32(gamma),
                       rows=rows)
    out = {"rows": int(len(rows)), "reference": "FP64 oracle (C, OpenMP) over all 2^20 sources"}
    for name, prec in (("fp32", None), ("fp16", "fp16"), ("bf16", "bf16")):
        y = y32 if prec is None else K.krr_kernel_mvp(X, q, sigma, gamma, prec=prec)
        yy = y.cpu().numpy().astype(np.float64)[rows]
        out[name] = float(np.max(np.abs(yy - ref) / scale))
    out["fp32_bar"] = 1e-5
    return out


def bench_config(world):
    """The workload both arms report (`config`)."""
    return {
        "workload": f"gaussian kernel product y=(K_hat+gamma I)q, N={MVP_N} uniform "
                    "unit cube d=3, sigma=0.05, gamma=1e-3, q~N(0,1), m=1; step = "
                    "prep (Morton sort, pack) + product + finalize through the C ABI",
        "l2": "512 MB buffer written between timed steps (inputs are 16 MB)",
        "parallelism": f"{world} independent problems (one per GPU)",
    }


def run_reference(args):
    # host-only: rank 0 times the oracle, the other ranks exit without work
    # (no process group is needed)
    if int(os.environ.get("RANK", "0")) != 0:
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
    sample = (f"{rows_per_step} seeded target rows x {MVP_N} sources per step (the FP64 oracle "
              "on the host cores; the rate is per evaluated pair, as on the GPU)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gpairs/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(int(os.environ.get("WORLD_SIZE", "1"))),
        "cpu_baseline": {"value": value, "unit": "Gpairs/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Gpairs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ libkrr ---
T_START = time.perf_counter()


def progress(msg):
    """One line on stderr per bench phase (the JSON line stays alone on stdout)."""
    sys.stderr.write(f"[bench {time.perf_counter() - T_START:7.1f} s] {msg}\n")
    sys.stderr.flush()


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
    ex2_f16x2, ex2_bf16x2, mma_sync_flops = K.krr_measure_half_rates()
    rates = {"ex2_f32_per_s": ex2_rate, "ex2_f16x2_values_per_s": ex2_f16x2,
             "ex2_bf16x2_values_per_s": ex2_bf16x2, "fp32_lanes_per_s": fp32_lanes,
             "mma_sync_m16n8k16_f16_flops_per_s": mma_sync_flops}

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
    # CUDA-core work per pair of the product's path (expanded form): one
    # MUFU.EX2, plus d + 1 FP32 operations when the exponent is formed on the
    # CUDA cores, or 1 (the weighted accumulate) when the tensor cores form it
    tensor_exp = prof["tensor_exponent_launches"] == prof["product_launches"] > 0
    fp32_per_pair = 1 if tensor_exp else MVP_D + 1
    peak_pairs = min(ex2_rate, fp32_lanes / fp32_per_pair)
    kernel_name = ("mvp_tcx_kernel (exponent on the tensor cores) + direct-form tail"
                   if tensor_exp else "mvp_f32_kernel")

    progress(f"headline product: {value:.0f} Gpairs/s")
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
    # the same on the other kernels (handle option KRR_OPT_TCGEN05): the
    # mma.sync kernel, and the kernel with the exponent in tensor memory
    m16_alt = {}
    for name, opt in (("mma_sync_ms", 0), ("tmem_exponent_ms", 2)):
        h5 = K.Handle()
        K.krr_set_option(K.KRR_OPT_TCGEN05, opt, handle=h5)
        K.krr_kernel_mvp(X, Q16, sigma, gamma, out=Y16, handle=h5)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        K.krr_kernel_mvp(X, Q16, sigma, gamma, out=Y16, handle=h5)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        m16_alt[name] = e0.elapsed_time(e1)
        h5.close()

    progress(f"16-column product: {m16_ms:.1f} ms (mma.sync kernel {m16_alt['mma_sync_ms']:.1f} ms, "
             f"tensor-memory exponent kernel {m16_alt['tmem_exponent_ms']:.1f} ms)")
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

    # ---- FP64 oracle on the host cores (rank 0, one GPU only)
    cpu = None
    errors = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nrows = 32768  # about 10 s of the oracle on 16 cores
        rows = inputs.sample_rows(MVP_N, nrows, seed=11)
        rate, dt, cores, ref = cpu_oracle_rate(p["X"], p["Q"], sigma, gamma, rows, with_values=True)
        cpu = {"value": rate, "unit": "Gpairs/s", "cores": cores, "kind": "oracle",
               "sample": f"{nrows} seeded target rows x {MVP_N} sources ({dt:.1f} s)"}
        # the products' error against these oracle sums (every 8th sampled row)
        sub = np.arange(0, nrows, 8)
        errors = precision_errors(K, X, q, y, sigma, gamma, p, rows[sub], ref[sub])
        cpu["solves_2000pt_2d"] = cpu_oracle_solves(inputs.small_problem(seed=0))

    progress("end-to-end and CPU baseline done")
    # ---- FGMRES time to a 1e-6 relative residual: the plain FP32 form next
    # to the precision, block (many right-hand sides) and batching forms, the
    # gradient, and the Matern / high-d / autotune extras.  They run on one
    # GPU only (a multi-GPU run measures the product) and in this order while
    # the wall-clock budget lasts; a skipped form is recorded as such.
    solve, grad, matern, tuned, highd, latency = {}, None, None, None, None, None
    skipped = []
    extras = world == 1
    sharded = sharded_product(K, torch, inputs, rank, world, dev, stream) if world > 1 else None

    def budget_left(name):
        el = time.perf_counter() - T_START
        if el <= args.budget_s:
            progress(f"{name} (at {el:.0f} s)")
            return True
        skipped.append(name)
        return False

    if extras:
        sp = inputs.small_problem(seed=rank)
        solve["small_2000pt_2d"] = {"fgmres": solve_once(K, torch, sp, dev, stream, "fp32"),
                                    "cg": cg_once(K, torch, sp, dev, stream),
                                    "fcg": fcg_once(K, torch, sp, dev, stream)}
        if args.batch_probs > 0 and budget_left("batching_d8"):
            solve["batching_d8"] = batching_form(K, torch, inputs, args, rank, dev, stream)
        if args.precision_n > 0 and budget_left("precision_full"):
            solve[f"precision_mixture_{args.precision_n}pt_2d"] = precision_full(K, torch, inputs, args,
                                                                                  rank, dev, stream)
        if args.grad_n > 0 and budget_left("mll_grad"):
            grad = gradient_form(K, torch, inputs, args, rank, dev, stream)
        if args.solve_n > 0 and budget_left("mixture_forms"):
            solve[f"mixture_forms_{args.solve_n}pt_2d"] = mixture_forms(K, torch, inputs, args, rank, dev,
                                                                        stream)
        if args.highd and budget_left("highd"):
            highd = highd_form(K, torch, rank, dev, ex2_rate)
        if args.matern and budget_left("matern"):
            matern = matern_form(K, torch, inputs, X, q, rank, dev, stream, ex2_rate, fp32_lanes)
        if args.autotune and budget_left("autotune"):
            tuned = autotune_form(K, torch, inputs, args, X, q, Q16, sigma, gamma, rank, dev, stream,
                                  kern_ms, m16_ms)
        if budget_left("small_product_latency"):
            latency = small_product_latency(K, torch, rank, dev)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gpairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(world),
            "roofline": {
                "bound": "alu", "achieved": achieved, "peak": peak_pairs / 1e9,
                "unit": "Gpairs/s", "frac": achieved * 1e9 / peak_pairs,
                "traffic": traffic_bytes(tensor_exp),
                "kernel": kernel_name, "launch_ms": kern_ms,
                "peak_source": "measured on this GPU: min(MUFU.EX2 rate, FP32 lane rate / FP32 "
                               f"operations per pair) = min({ex2_rate / 1e12:.2f}e12, "
                               f"{fp32_lanes / 1e12:.2f}e12/{fp32_per_pair})",
            },
            "e2e": {"value": e2e_value, "unit": "Gpairs/s",
                    "h2d_bytes_per_step": MVP_N * (MVP_D + 1) * 4, "d2h_bytes_per_step": MVP_N * 4},
            "gpu_launches": launches,
            "clocks": clk,
            "mvp_m16": {"ms": m16_ms, "Gpair_rhs_per_s": pairs * 16 / (m16_ms / 1e3) / 1e9,
                        "kernel": "mvp_umx_kernel (exponent by mma.sync, P Q by tcgen05; default "
                                  "for float32 products of more than 8 columns)",
                        **m16_alt},
            "fgmres": solve,
            "skipped_for_wall_budget": skipped,
            "rates": rates,
            "mll_grad": grad,
            "matern": matern,
            "autotune": tuned,
            "small_product_latency": latency,
            "highd": highd,
            "sharded_product": sharded,
            "cpu_baseline": cpu,
            "precision_errors": errors,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def traffic_bytes(tensor_exp):
    """ncu DRAM bytes of one product (all its kernels) on this workload, or
    None once a kernel source changed since the capture."""
    import hashlib
    t = TRAFFIC_TCX if tensor_exp else TRAFFIC
    for src, sha in t["sources"].items():
        try:
            h = hashlib.sha1(open(os.path.join(ROOT, src), "rb").read()).hexdigest()
        except OSError:
            return None
        if h != sha:
            return None
    return t["bytes"]


def solve_once(K, torch, p, dev, stream, inner_prec, handle=None):
    """Time one FGMRES solve (prep included) with CUDA events; FP64-recheck
    is left to the tests.  Returns a report dict."""
    X = torch.from_numpy(p["X"]).to(dev)
    b = torch.from_numpy(p["b"]).to(dev)
    opts = K.default_opts(delta=p["delta"], inner_tol=p["inner_tol"], restart=p["restart"],
                          tol=p["tol"], inner_prec=inner_prec)
    warm = K.default_opts(restart=p["restart"], max_cycles=1, inner_maxit=1,
                          inner_prec=inner_prec)
    K.krr_fgmres_solve(X, b, p["sigma"], p["gamma"], opts=warm, handle=handle)  # allocates the workspace
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    x, info = K.krr_fgmres_solve(X, b, p["sigma"], p["gamma"], opts=opts, handle=handle)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    i = info[0]
    return {"time_to_solution_ms": e0.elapsed_time(e1), "relres_true": i["relres_true"],
            "outer": i["outer_iters"], "inner": i["inner_iters"], "cycles": i["cycles"],
            "status": K.status_string(i["status"]), "inner_prec": inner_prec,
            "N": int(p["X"].shape[0])}


def _timed(torch, stream, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1)


def _report(K, infos):
    return {"relres_true_max": max(i["relres_true"] for i in infos),
            "outer_max": max(i["outer_iters"] for i in infos),
            "inner_max": max(i["inner_iters"] for i in infos),
            "all_ok": all(i["status"] == K.KRR_OK for i in infos)}


def cg_once(K, torch, p, dev, stream, handle=None):
    X = torch.from_numpy(p["X"]).to(dev)
    b = torch.from_numpy(p["b"]).to(dev)
    K.krr_cg_solve(X, b, p["sigma"], p["gamma"], tol=1e-6, maxit=1, handle=handle)  # workspace
    (x, info), ms = _timed(torch, stream, lambda: K.krr_cg_solve(X, b, p["sigma"], p["gamma"],
                                                                 tol=1e-6, maxit=20000,
                                                                 handle=handle))
    return {"time_to_solution_ms": ms, "relres_true": info["relres_true"],
            "iters": info["outer_iters"], "status": K.status_string(info["status"])}


def fcg_once(K, torch, p, dev, stream):
    """Flexible CG with the paper's flexible-CG settings (delta = inner tol =
    1e-4, window 30)."""
    X = torch.from_numpy(p["X"]).to(dev)
    b = torch.from_numpy(p["b"]).to(dev)
    opts = K.default_opts(delta=1e-4, inner_tol=1e-4, inner_maxit=2000, restart=30)
    K.krr_fcg_solve(X, b, p["sigma"], p["gamma"], opts=K.default_opts(max_cycles=1, restart=1,
                                                                     inner_maxit=1))  # workspace
    (x, info), ms = _timed(torch, stream, lambda: K.krr_fcg_solve(X, b, p["sigma"], p["gamma"], opts=opts))
    i = info[0]
    return {"time_to_solution_ms": ms, "relres_true": i["relres_true"], "outer": i["outer_iters"],
            "inner": i["inner_iters"], "status": K.status_string(i["status"])}


def sharded_product(K, torch, inputs, rank, world, dev, stream, reps=3):
    """On N > 1 GPUs: ONE 2^20-point product (the headline problem, seed 0 on
    every rank) with its target rows split over the ranks, each rank summing
    N^2 / world pairs and a sum all-reduce (NCCL) assembling y on every rank
    (paper_1408_1237_gb300/distributed.py).  Strong scaling: the reported
    rate is N^2 pairs over the slowest rank's time per product, collective
    included."""
    from paper_1408_1237_gb300 import distributed
    p = inputs.mvp_problem(seed=0, N=MVP_N, d=MVP_D)
    X = torch.from_numpy(p["X"]).to(dev)
    q = torch.from_numpy(p["Q"]).to(dev)
    distributed.sharded_kernel_mvp(X, q, p["sigma"], p["gamma"])
    barrier(world, dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(reps):
        distributed.sharded_kernel_mvp(X, q, p["sigma"], p["gamma"])
    torch.cuda.synchronize(dev)
    t = max_over_ranks((time.perf_counter() - t0) / reps, world, dev)
    return {"ranks": world, "ms_per_product": t * 1e3,
            "Gpairs_per_s": float(MVP_N) * MVP_N / t / 1e9, "scaling": "strong",
            "collective_bytes_per_rank": distributed.collective_bytes_per_rank(MVP_N, 1, world)}


def mixture_opts(K, prec, cap, cycles=4, delta=1e-2):
    """Solver settings of the precision form: delta = 10 gamma (Sec. 6), inner
    tolerance 1e-2, restart 30, outer tolerance 1e-6, at most `cycles`
    restart cycles (a form that stalls is reported unconverged, not run on)."""
    return K.default_opts(delta=delta, inner_tol=1e-2, inner_maxit=cap, restart=30, max_cycles=cycles,
                          inner_prec=prec)


def precision_full(K, torch, inputs, args, rank, dev, stream):
    """The precision-form configuration at full size: 262,144 points of the
    16-component mixture (sigma 0.03, gamma 1e-3), b = smooth field plus
    N(0, 0.01^2) noise, FGMRES with the truncated-CG preconditioner and
    float32 inner products, to a true relative residual of 1e-6 (reported by
    the library's accurate product; the tests recheck such solutions with the
    FP64 oracle)."""
    mp = inputs.mixture_problem(seed=rank, N=args.precision_n)
    X = torch.from_numpy(mp["X"]).to(dev)
    b = torch.from_numpy(mp["b"]).to(dev)
    K.krr_fgmres_solve(X, b, mp["sigma"], mp["gamma"], opts=K.default_opts(max_cycles=1, inner_maxit=1))
    (x, info), ms = _timed(torch, stream, lambda: K.krr_fgmres_solve(
        X, b, mp["sigma"], mp["gamma"], opts=mixture_opts(K, "fp32", args.precision_cap, cycles=2)))
    i = info[0]
    return {"N": args.precision_n, "form": "plain FP32 inner, single right-hand side",
            "delta": 1e-2, "inner_tol": 1e-2, "inner_cap": args.precision_cap,
            "time_to_solution_ms": ms, "relres_true": i["relres_true"], "outer": i["outer_iters"],
            "inner": i["inner_iters"], "status": K.status_string(i["status"])}


def mixture_forms(K, torch, inputs, args, rank, dev, stream):
    """Every form on the mixture cloud at --solve-n points (kernel sigma 0.03,
    gamma 1e-3, delta = 10 gamma, inner tol 1e-2, restart 30): the paper's
    right-hand side b (smooth field plus noise) solved alone with float32
    and f16 inner products, and 16 right-hand sides (b and 15 N(0,1)
    columns) per RHS: single-column float32 solves of the first plain-cols
    columns against 16-column lockstep blocks with float32 and f16 inner
    products."""
    import numpy as np
    mp = inputs.mixture_problem(seed=rank, N=args.solve_n)
    rng = np.random.default_rng(100 + rank)
    B = np.stack([mp["b"]] + [rng.standard_normal(args.solve_n).astype(np.float32) for _ in range(15)])
    X = torch.from_numpy(mp["X"]).to(dev)
    Bd = torch.from_numpy(B).to(dev)
    out = {"N": args.solve_n, "inner_cap": args.solve_cap}
    cap = args.solve_cap
    K.krr_fgmres_solve(X, Bd[0].contiguous(), mp["sigma"], mp["gamma"],
                       opts=K.default_opts(max_cycles=1, inner_maxit=1))  # workspace
    for prec, cyc in (("fp32", 4), ("fp16", 2)):
        (x, info), ms = _timed(torch, stream, lambda: K.krr_fgmres_solve(
            X, Bd[0].contiguous(), mp["sigma"], mp["gamma"], opts=mixture_opts(K, prec, cap, cyc)))
        out[f"b_{prec}_inner"] = dict(time_to_solution_ms=ms, **_report(K, info))
    ms_all, infos = [], []
    for c in range(min(args.plain_cols, 16)):
        (x, info), ms = _timed(torch, stream, lambda: K.krr_fgmres_solve(
            X, Bd[c].contiguous(), mp["sigma"], mp["gamma"], opts=mixture_opts(K, "fp32", cap)))
        ms_all.append(ms)
        infos += info
    out["plain_fp32"] = dict(per_rhs_ms=sum(ms_all) / len(ms_all), rhs_timed=len(ms_all), **_report(K, infos))
    for form, prec in (("block16_fp32", "fp32"), ("block16_fp16_inner", "fp16")):
        (x, infos), ms = _timed(torch, stream, lambda: K.krr_fgmres_solve(
            X, Bd, mp["sigma"], mp["gamma"], opts=mixture_opts(K, prec, cap, cycles=3 if prec == "fp32" else 2)))
        out[form] = dict(total_ms=ms, per_rhs_ms=ms / 16, **_report(K, infos))
    plain = out["plain_fp32"]["per_rhs_ms"]
    for form in ("block16_fp32", "block16_fp16_inner"):
        out[form]["speedup_vs_plain_fp32"] = plain / out[form]["per_rhs_ms"]
    out["b_fp16_inner"]["speedup_vs_fp32_inner"] = (out["b_fp32_inner"]["time_to_solution_ms"] /
                                                    out["b_fp16_inner"]["time_to_solution_ms"])
    return out


def batch_opts(K, prec):
    """Solver settings of the batching form: delta = 10 gamma_k (Sec. 6),
    inner tolerance 1e-2, at most 400 inner steps, restart 30, at most 8
    restart cycles."""
    return K.default_opts(inner_tol=1e-2, inner_maxit=400, restart=30, max_cycles=8, inner_prec=prec)


def batching_form(K, torch, inputs, args, rank, dev, stream, handle=None, plain=True):
    """The batching workload (d = 8, N(0, I) points, sigma 1, gamma
    log-uniform in [1e-4, 1e-1], 16 N(0,1) right-hand sides each, N
    log-uniform in [1024, batch-nmax]): all problems in one batched call
    (float32 inner products by default; --batch-fp16 adds the f16-inner
    call) against the plain float32 form: single-column
    solves, one right-hand side of each problem of a seeded sample of
    batch-plain problems; its per-RHS time is the sample mean, an unbiased
    estimate of the mean over all problems."""
    import numpy as np
    bp = inputs.batch_problems(seed=rank, nprob=args.batch_probs, d=8, m=16, n_lo=1024,
                               n_hi=args.batch_nmax)
    probs = []
    for pr in bp["problems"]:
        N = pr["X"].shape[0]
        probs.append(dict(X=torch.from_numpy(pr["X"]).to(dev),
                          B=torch.from_numpy(np.ascontiguousarray(pr["B"].T)).to(dev),
                          gamma=pr["gamma"],
                          Xsol=torch.empty((16, N), dtype=torch.float64, device=dev)))
    nrhs = 16 * len(probs)
    out = {"problems": len(probs), "N_min": int(min(p["X"].shape[0] for p in probs)),
           "N_max": int(max(p["X"].shape[0] for p in probs)),
           "pairs_per_sweep": float(sum(float(p["X"].shape[0]) ** 2 for p in probs)),
           "rhs_per_problem": 16}
    first_ms = None
    if handle is not None:  # the first call tunes every product shape of the batch
        _, first_ms = _timed(torch, stream, lambda: K.krr_fgmres_solve_batched(
            probs, d=8, sigma=bp["sigma"], m_rhs=16, opts=batch_opts(K, "fp16"), handle=handle))
    for form, prec in args.batch_forms:
        infos, ms = _timed(torch, stream, lambda: K.krr_fgmres_solve_batched(
            probs, d=8, sigma=bp["sigma"], m_rhs=16, opts=batch_opts(K, prec), handle=handle))
        out[form] = dict(total_ms=ms, per_rhs_ms=ms / nrhs, **_report(K, infos))
        if first_ms is not None:
            out[form]["first_call_ms"] = first_ms
            first_ms = None
        if not plain:
            return out
    rng = np.random.default_rng(500 + rank)
    sample = sorted(rng.choice(len(probs), size=min(args.batch_plain, len(probs)), replace=False).tolist())
    tot, pinfos = 0.0, []
    for k in sample:
        pr = probs[k]
        (x, info), ms1 = _timed(torch, stream, lambda: K.krr_fgmres_solve(
            pr["X"], pr["B"][0].contiguous(), bp["sigma"], pr["gamma"], opts=batch_opts(K, "fp32")))
        tot += ms1
        pinfos += info
    out["plain_fp32"] = dict(per_rhs_ms=tot / len(sample), sampled_problems=sample,
                             estimated_total_ms=tot / len(sample) * nrhs, **_report(K, pinfos))
    for form, _ in args.batch_forms:
        out[form]["speedup_vs_plain_fp32"] = out["plain_fp32"]["per_rhs_ms"] / out[form]["per_rhs_ms"]
    return out


def gradient_form(K, torch, inputs, args, rank, dev, stream):
    """Log-marginal-likelihood gradient (log sigma, log gamma, X) with 32
    Rademacher probes on the uniform 4-D cloud (sigma 0.2, gamma 1e-2): the
    33 right-hand sides solve as lockstep blocks, then the adjoint kernel."""
    gp = inputs.gradient_problem(seed=rank, N=args.grad_n, d=4, probes=32)
    X = torch.from_numpy(gp["X"]).to(dev)
    y = torch.from_numpy(gp["y"]).to(dev)
    (gs, gg, gX, infos), ms = _timed(torch, stream, lambda: K.krr_mll_grad(
        X, y, gp["sigma"], gp["gamma"], n_probes=32, seed=gp["seed"]))
    return dict(N=args.grad_n, d=4, probes=32, time_ms=ms, dlogsigma=gs, dloggamma=gg, **_report(K, infos))


def matern_form(K, torch, inputs, X, q, rank, dev, stream, ex2_rate, fp32_lanes):
    """The Matern kernel (Sec. 6.1, smoothness 3/2) on its own handle: the
    single-column product on the 2^20-point cube (h = 0.1) against its ALU
    roofline, and time to a 1e-6 residual on the 2000-point problem and on
    two-class clouds shaped like the paper's Matern table (N = 1000)."""
    h = K.Handle()
    K.krr_set_option(K.KRR_OPT_KERNEL, K.KRR_KERNEL_MATERN32, handle=h)
    hl, gamma = 0.1, 1e-3
    y = torch.empty_like(q)
    K.krr_kernel_mvp(X, q, hl, gamma, out=y, handle=h)
    rsqrt_rate = K.krr_measure_rsqrt_rate(handle=h)
    torch.cuda.synchronize(dev)
    K.krr_profile_enable(True, handle=h)
    reps = 3
    (_, ms) = _timed(torch, stream, lambda: [K.krr_kernel_mvp(X, q, hl, gamma, out=y, handle=h)
                                             for _ in range(reps)])
    prof = K.krr_profile_read(handle=h)
    K.krr_profile_enable(False, handle=h)
    n = X.shape[0]
    pairs = float(n) * n
    kern_ms = prof["product_ms"] / max(prof["product_launches"], 1)
    # direct form per pair: d differences, d multiply-adds, three multiplies
    # (r = r^2 rsqrt(r^2), a = s r, the exponent), the (1 + a) e FMA and the
    # weighted accumulate on the FP32 lanes; one rsqrt and one EX2 on MUFU
    d = X.shape[1]
    fp32_ops = 2 * d + 5
    peak = min(fp32_lanes / fp32_ops, 1.0 / (1.0 / ex2_rate + 1.0 / rsqrt_rate))
    product = {"N": n, "d": d, "h": hl, "step_ms": ms / reps, "kernel_ms": kern_ms,
               "Gpairs_per_s": pairs / (kern_ms / 1e3) / 1e9,
               "roofline": {"bound": "alu", "peak_Gpairs_per_s": peak / 1e9,
                            "frac": pairs / (kern_ms / 1e3) / peak,
                            "peak_source": f"min(FP32 lanes {fp32_lanes / 1e12:.2f}e12 / {fp32_ops}, "
                                           f"1 / (1/EX2 {ex2_rate / 1e12:.2f}e12 + 1/rsqrt "
                                           f"{rsqrt_rate / 1e12:.2f}e12))",
                            "kernel": "mvp_f32_kernel<3, 8, Matern> (direct form, 8 targets per thread)"}}
    solves = {}
    sp = inputs.small_problem(seed=rank)
    sp = dict(sp, sigma=0.1)  # h = 0.1 on the 2000-point problem
    solves["small_2000pt_2d"] = {"fgmres": solve_once(K, torch, sp, dev, stream, "fp32", handle=h),
                                 "cg": cg_once(K, torch, sp, dev, stream, handle=h)}
    for dd in (3, 14, 25, 61):
        mp = inputs.matern_problem(seed=rank + dd, N=1000, d=dd)
        solves[f"classification_1000pt_d{dd}"] = {
            "fgmres": solve_once(K, torch, mp, dev, stream, "fp32", handle=h),
            "cg": cg_once(K, torch, mp, dev, stream, handle=h)}
    h.close()
    return {"product": product, "solves": solves}


def autotune_form(K, torch, inputs, args, X, q, Q16, sigma, gamma, rank, dev, stream, kern_ms, m16_ms):
    """Products and the batching subset on a handle with KRR_OPT_AUTOTUNE: the
    first call of each shape tunes its source splits (timed separately), the
    next ones run the tuned plan."""
    h = K.Handle()
    K.krr_set_option(K.KRR_OPT_AUTOTUNE, 1, handle=h)
    y = torch.empty_like(q)
    Y16 = torch.empty_like(Q16)
    (_, tune1_ms) = _timed(torch, stream, lambda: K.krr_kernel_mvp(X, q, sigma, gamma, out=y, handle=h))
    (_, tune16_ms) = _timed(torch, stream, lambda: K.krr_kernel_mvp(X, Q16, sigma, gamma, out=Y16, handle=h))
    K.krr_profile_enable(True, handle=h)
    reps = 3
    for _ in range(reps):
        K.krr_kernel_mvp(X, q, sigma, gamma, out=y, handle=h)
    prof = K.krr_profile_read(handle=h)
    K.krr_profile_enable(False, handle=h)
    t1 = prof["product_ms"] / max(prof["product_launches"], 1)
    (_, t16) = _timed(torch, stream, lambda: K.krr_kernel_mvp(X, Q16, sigma, gamma, out=Y16, handle=h))
    out = {"product_m1": {"model_kernel_ms": kern_ms, "tuned_kernel_ms": t1, "first_call_ms": tune1_ms},
           "product_m16": {"model_ms": m16_ms, "tuned_ms": t16, "first_call_ms": tune16_ms}}
    if args.batch_probs > 0:
        # a 4-problem subset (N <= 8192) of the batching workload: the first
        # call tunes each branch's product shapes
        sub = argparse.Namespace(**vars(args))
        sub.batch_probs, sub.batch_nmax = 4, 8192
        out["batching_subset_4x8192"] = batching_form(K, torch, inputs, sub, rank, dev, stream, handle=h,
                                                      plain=False)
    h.close()
    return out


def small_product_latency(K, torch, rank, dev, N=4096, reps=200):
    """Latency of one small single-column product (N = 4096 uniform points in
    the unit cube, d = 3), device arrays, mean over `reps` back-to-back calls
    between two synchronisations: krr_kernel_mvp (prepares the points and
    waits for their block counts every call), krr_kernel_mvp_points on a
    prepared point set (no host synchronisation), and the same product
    captured once in a CUDA graph and replayed."""
    import numpy as np
    rng = np.random.default_rng(4242 + rank)
    X = torch.from_numpy(rng.random((N, 3)).astype(np.float32)).to(dev)
    q = torch.from_numpy(rng.standard_normal(N).astype(np.float32)).to(dev)
    y = torch.empty_like(q)
    h = K.Handle()
    out = {"N": N, "d": 3, "reps": reps}
    try:
        def timed(fn):
            fn()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for _ in range(reps):
                fn()
            torch.cuda.synchronize(dev)
            return (time.perf_counter() - t0) / reps * 1e6
        out["kernel_mvp_us"] = timed(lambda: K.krr_kernel_mvp(X, q, 0.05, 1e-3, out=y, handle=h))
        P = K.Points(X, 0.05, handle=h)
        try:
            out["points_us"] = timed(lambda: K.krr_kernel_mvp_points(P, q, 1e-3, out=y))
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                K.krr_kernel_mvp_points(P, q, 1e-3, out=y)
            out["graph_replay_us"] = timed(g.replay)
        finally:
            P.close()
    finally:
        h.close()
    return out


def tensor_peak_tflops():
    """Measured dense bf16 tensor peak of this machine (burst), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def highd_form(K, torch, rank, dev, ex2_rate):
    """High-dimensional single-column products (N = 65536 uniform in [0,1]^d):
    the cross term on the tensor cores (kernel width 0.3 sqrt(d): compact
    super-blocks), with tcgen05 (default) and with mma.sync (option), against
    the direct form on the CUDA cores (the same points at width 0.02 sqrt(d):
    no compact block).  Rooflines per kernel: the algorithmic contraction is
    the cross term, 2 d flops per pair (against the dense bf16 peak), and
    every pair takes one MUFU.EX2 (against the EX2 rate measured live); the
    kernel issues 3 (d + 1) split-f16 products per pair (`issued_tflops`),
    which is work of the float32-grade split, not of the method."""
    import numpy as np
    peak, src = tensor_peak_tflops()
    out = {}
    for d in (16, 32, 64):
        rng = np.random.default_rng(1000 + 17 * rank + d)
        n = 65536
        X = torch.from_numpy(rng.random((n, d)).astype(np.float32)).to(dev)
        q = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(dev)
        y = torch.empty_like(q)
        row = {}
        for name, width, tc5 in (("tensor", 0.3, 0), ("tcgen05", 0.3, 1), ("direct", 0.02, 1)):
            sig = width * float(np.sqrt(d))
            h = K.Handle()
            K.krr_set_option(K.KRR_OPT_HIGHD_TCGEN05, tc5, handle=h)
            K.krr_kernel_mvp(X, q, sig, 1e-3, out=y, handle=h)
            torch.cuda.synchronize(dev)
            K.krr_profile_enable(True, handle=h)
            for _ in range(3):
                K.krr_kernel_mvp(X, q, sig, 1e-3, out=y, handle=h)
            prof = K.krr_profile_read(handle=h)
            h.close()
            ms = prof["product_ms"] / max(prof["product_launches"], 1)
            row[name] = {"kernel_ms": ms, "Gpairs_per_s": float(n) * n / ms / 1e6,
                         "tensor_path": prof["tensor_exponent_launches"] == prof["product_launches"]}
        kname = {"tensor": f"mvp_tch_kernel<{((d + 15) // 16) * 16}> (mma.sync m16n8k16, by option)",
                 "tcgen05": f"mvp_uhd_kernel<{((d + 15) // 16) * 16}> (tcgen05.mma, TMEM)"}
        for name in ("tensor", "tcgen05"):
            pairs_s = float(n) * n / (row[name]["kernel_ms"] / 1e3)
            tflops = pairs_s * 2 * d / 1e12
            row[name]["roofline"] = {"bound": "tensor", "achieved": tflops, "peak": peak,
                                     "unit": "TFLOP/s", "frac": tflops / peak,
                                     "peak_source": f"bf16 dense, {src}",
                                     "flops_per_pair": 2 * d, "kernel": kname[name]}
            row[name]["ex2_roofline"] = {"bound": "alu", "achieved": pairs_s / 1e9,
                                         "peak": ex2_rate / 1e9, "unit": "Gpairs/s",
                                         "frac": pairs_s / ex2_rate,
                                         "peak_source": "MUFU.EX2 rate measured on this GPU, 1 per pair"}
            row[name]["issued_tflops"] = pairs_s * 2 * 3 * (d + 1) / 1e12
        row["speedup_mma_sync"] = row["direct"]["kernel_ms"] / row["tensor"]["kernel_ms"]
        row["speedup"] = row["direct"]["kernel_ms"] / row["tcgen05"]["kernel_ms"]
        out[f"d{d}"] = row
    return out


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_libkrr(args)


if __name__ == "__main__":
    sys.exit(main())
