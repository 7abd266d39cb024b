"""Row-sharded kernel product across the ranks of a torch.distributed group.

The product y = (K_hat + gamma I) q is the O(N^2) step that the paper runs
on the GPU (Sec. 3.1); split over P ranks by target rows, each rank sums its
rows against all sources (N^2 / P pairs) and one collective assembles y on
every rank before the next Krylov step.  Rank k computes the Morton-ordered
super-blocks [k nsb / P, (k+1) nsb / P) of 256 targets (the library's
KRR_OPT_SHARD_COUNT / KRR_OPT_SHARD_INDEX), writing its rows into a zeroed Y;
the collective is a sum all-reduce of Y (rows a rank did not compute are
exact zeros, so the sum reassembles the unsharded product bit for bit).  In
original row order a shard's rows are scattered, so the sum replaces an
all-gather: a ring all-reduce moves 2 (P-1)/P x 4 N m bytes per rank.

The collective is torch.distributed plumbing: NCCL for device tensors on an
NCCL group, or gloo, through host memory, when the group's backend is gloo.
Every kernel of the product runs in libkrr; this module only sets the shard
options, zero-fills the output and calls the collective.
"""
from . import binding


def _all_reduce_sum(t, group):
    import torch
    import torch.distributed as dist
    if t.is_cuda and dist.get_backend(group) == "gloo":
        host = t.cpu()
        dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
        t.copy_(host)
        torch.cuda.current_stream(t.device).synchronize()
    else:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)


def sharded_kernel_mvp(X, Q, sigma, gamma, prec="fp32", group=None, handle=None, stream=None):
    """Y = (K_hat + gamma I) Q with the target rows split over the ranks of
    `group`: this rank computes its shard through the library, then a sum
    all-reduce gives every rank the whole Y.  X, Q as for
    binding.krr_kernel_mvp (the same arrays on every rank); torch tensors or
    NumPy arrays.  Returns Y like Q."""
    import numpy as np
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    h = handle or binding.default_handle()
    if isinstance(Q, np.ndarray):
        Y = np.zeros_like(Q, dtype=np.float32)
    else:
        Y = torch.zeros_like(Q, dtype=torch.float32)
    binding.krr_set_option(binding.KRR_OPT_SHARD_COUNT, world, handle=h)
    binding.krr_set_option(binding.KRR_OPT_SHARD_INDEX, rank, handle=h)
    try:
        binding.krr_kernel_mvp(X, Q, sigma, gamma, prec=prec, out=Y, handle=h, stream=stream)
    finally:
        binding.krr_set_option(binding.KRR_OPT_SHARD_COUNT, 1, handle=h)
        binding.krr_set_option(binding.KRR_OPT_SHARD_INDEX, 0, handle=h)
    if stream is not None and not isinstance(Y, np.ndarray) and not isinstance(stream, int):
        # the collective runs after torch's current stream: order it after the product
        torch.cuda.current_stream(Y.device).wait_stream(stream)
    _all_reduce_sum(torch.from_numpy(Y) if isinstance(Y, np.ndarray) else Y, group)
    return Y


def collective_bytes_per_rank(N, m, world):
    """Bytes one rank sends in the ring all-reduce of a float32 N x m output."""
    return 0 if world <= 1 else int(2 * (world - 1) * 4 * N * m // world)
