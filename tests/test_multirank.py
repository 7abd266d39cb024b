"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

On N GPUs every rank solves its own seeded problem (weak scaling); ranks
exchange only timings: a barrier and a MAX all-reduce of the elapsed time,
and the whole-job rate is all ranks' pairs over the slowest rank's time.
The reference arm (the FP64 oracle on the host) runs on rank 0 alone.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import bench
rank, world, local = bench.dist_setup(2)
assert world == 2 and rank == int(os.environ["RANK"])
bench.barrier(world, None)
t = bench.max_over_ranks(1.5 + rank, world, None)
rate = bench.whole_job_rate(1e9, world, t)
print(json.dumps({"rank": rank, "max_t": t, "rate": rate}))
import torch.distributed as dist
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, port):
    env = dict(os.environ)
    env.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(port), KRR_BENCH_BACKEND="gloo", CUDA_VISIBLE_DEVICES="")
    return env


def test_timing_exchange_two_ranks():
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", RANK_SCRIPT, ROOT], env=_env(r, port),
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        # the slowest rank's time, and both ranks' pairs over it
        assert o["max_t"] == 2.5
        assert o["rate"] == pytest.approx(2 * 1e9 / 2.5 / 1e9)


def test_reference_arm_rank0_only():
    port = _free_port()
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    procs = [subprocess.Popen(cmd, env=_env(r, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, cwd=ROOT) for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=600)
        assert p.returncode == 0, err
        outs.append(out.strip())
    assert outs[1] == ""
    line = json.loads(outs[0].splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


SHARD_SCRIPT = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch.distributed as dist
import oracle
from paper_1408_1237_gb300 import binding, distributed
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()

# a stand-in for the library on this GPU-less host: the shard options select
# rows [k N / P, (k+1) N / P), computed by the FP64 oracle and rounded to
# float32; rows outside the shard are left as they were
state = {"count": 1, "index": 0, "calls": 0}
def set_option(opt, value, handle=None):
    if opt == binding.KRR_OPT_SHARD_COUNT: state["count"] = value
    if opt == binding.KRR_OPT_SHARD_INDEX: state["index"] = value
def kernel_mvp(X, Q, sigma, gamma, prec="fp32", out=None, handle=None, stream=None):
    state["calls"] += 1
    N = X.shape[0]
    lo = N * state["index"] // state["count"]; hi = N * (state["index"] + 1) // state["count"]
    X64 = X.astype(np.float64)
    for c in range(Q.shape[0] if Q.ndim == 2 else 1):
        q = (Q[c] if Q.ndim == 2 else Q).astype(np.float64)
        y = oracle.mvp_rect(X64[lo:hi], X64, q, sigma) + gamma * q[lo:hi]
        (out[c] if Q.ndim == 2 else out)[lo:hi] = y.astype(np.float32)
    return out
binding.krr_set_option = set_option
binding.krr_kernel_mvp = kernel_mvp

rng = np.random.default_rng(3)
N, d, m = 1001, 3, 2
X = rng.random((N, d)).astype(np.float32)
Q = rng.standard_normal((m, N)).astype(np.float32)
Y = distributed.sharded_kernel_mvp(X, Q, 0.2, 1e-2, handle=object())
full = np.zeros_like(Q)
state.update(count=1, index=0)
kernel_mvp(X, Q, 0.2, 1e-2, out=full)
print(json.dumps({"rank": rank, "equal": bool(np.array_equal(Y, full)),
                  "reset": [state["count"], state["index"]],
                  "bytes": distributed.collective_bytes_per_rank(N, m, world)}))
dist.destroy_process_group()
"""


def test_sharded_product_collective_two_ranks():
    # the row-sharded product's host logic: shard options set and reset, the
    # zeroed output, and the sum all-reduce that gives every rank the whole y
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", SHARD_SCRIPT, ROOT], env=_env(r, port),
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["equal"], o
        assert o["reset"] == [1, 0]
        assert o["bytes"] == 2 * 1 * 4 * 1001 * 2 // 2
