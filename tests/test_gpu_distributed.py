"""Row-sharded product on two ranks that share this GPU (gloo, host staging).

Each of two processes computes its shard of the target rows through the
library and a gloo sum all-reduce (through host memory) assembles y; the two
processes' kernels are independent (neither waits on the other), so they may
share one GPU.  The assembled product must equal the unsharded one bit for
bit on both ranks, and match the FP64 oracle on sampled rows.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from conftest import f32

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import numpy as np, torch, torch.distributed as dist
from paper_1408_1237_gb300 import binding as K, distributed, inputs
dist.init_process_group("gloo")
rank = dist.get_rank()
out = {}
for name, (N, d, m, sigma) in {"cube": (60000, 3, 1, 0.05), "batch": (20000, 8, 16, 1.0)}.items():
    rng = np.random.default_rng(11)
    X = (rng.standard_normal((N, d)) if d == 8 else rng.random((N, d))).astype(np.float32)
    Q = rng.standard_normal((m, N) if m > 1 else N).astype(np.float32)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    Y = distributed.sharded_kernel_mvp(Xd, Qd, sigma, 1e-3).cpu().numpy()
    full = K.krr_kernel_mvp(Xd, Qd, sigma, 1e-3).cpu().numpy()
    np.save(os.path.join(sys.argv[2], f"{name}_{rank}.npy"), Y)
    out[name] = bool(np.array_equal(Y, full))
print(json.dumps({"rank": rank, "equal": out}))
dist.destroy_process_group()
"""


@pytest.fixture(scope="module")
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_share_gpu_sharded_product(built, oracle_mod, tmp_path):
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", RANK, ROOT, str(tmp_path)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=600)
        assert p.returncode == 0, err[-3000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["equal"] == {"cube": True, "batch": True}, o
    # both ranks hold the same y, and it matches the FP64 oracle on sampled rows
    from paper_1408_1237_gb300 import inputs
    for name, (N, d, m, sigma) in {"cube": (60000, 3, 1, 0.05), "batch": (20000, 8, 16, 1.0)}.items():
        Y0, Y1 = np.load(tmp_path / f"{name}_0.npy"), np.load(tmp_path / f"{name}_1.npy")
        assert np.array_equal(Y0, Y1)
        rng = np.random.default_rng(11)
        X = (rng.standard_normal((N, d)) if d == 8 else rng.random((N, d))).astype(np.float32)
        Q = rng.standard_normal((m, N) if m > 1 else N).astype(np.float32).reshape(m, N)
        rows = inputs.sample_rows(N, 128, seed=2)
        X64 = X.astype(np.float64)
        for c in range(min(m, 3)):
            q = Q[c].astype(np.float64)
            ref = oracle_mod.mvp(X64, q, f32(sigma), f32(1e-3), rows=rows)
            scale = oracle_mod.mvp(X64, np.abs(q), f32(sigma), f32(1e-3), rows=rows)
            assert np.max(np.abs(Y0.reshape(m, N)[c][rows] - ref) / scale) <= 1e-5
