"""Data-parallel training of one network over the ranks of a torch.distributed
process group: the collocation points are sharded, the weights replicated.

The loss of Section 4 (Eq. 4, Eq. 8) is a mean over points, so its value and
its weight gradient are sums of per-shard contributions.  Each rank computes
its shard's contributions with hrkan_train_step_partial (means over the
totals of all shards), the ranks sum them with one all-reduce of the gradient
(float32, P values) and one of the three float64 loss terms, and every rank
then applies the same adam_step: the replicas stay identical.  All arithmetic
of the step runs in the library's kernels; the all-reduce is the process
group's (NCCL between GPUs, gloo on the host).
"""
from __future__ import annotations

from . import capi


def shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """[begin, end) of rank's contiguous share of n points (shares differ by at most one)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"shard of {n} points for rank {rank} of {world}")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


class DataParallelStep:
    """The training step of one rank.  x_int [2, N_int], x_bnd [2, N_bnd] and
    g_bnd [N_bnd] are the whole point sets (the same on every rank); the rank
    keeps its shard of each."""

    def __init__(self, h, prob, x_int, x_bnd, g_bnd, group=None):
        import torch
        import torch.distributed as dist
        self.h, self.prob, self.group = h, prob, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.n_int_total, self.n_bnd_total = int(x_int.shape[1]), int(x_bnd.shape[1])
        a, b = shard(self.n_int_total, self.rank, self.world)
        c, d = shard(self.n_bnd_total, self.rank, self.world)
        self.x_int = x_int[:, a:b].contiguous()
        self.x_bnd = x_bnd[:, c:d].contiguous()
        self.g_bnd = g_bnd[c:d].contiguous()
        dev = x_int.device
        self.loss = torch.zeros(3, dtype=torch.float64, device=dev)
        self.dW = torch.zeros(int(h.P), dtype=torch.float32, device=dev)

    def __call__(self, W, lr, t, b1=0.9, b2=0.999, eps=1e-8):
        """One step at Adam step t >= 1: W (the replica's weights) is updated in place; returns
        the loss terms [L, mean r^2, mean (u-g)^2] at W before the update."""
        import torch.distributed as dist
        capi.hrkan_train_step_partial(self.h, self.prob, W, self.x_int, self.x_int.shape[1], self.x_bnd,
                                      self.g_bnd, self.x_bnd.shape[1], self.n_int_total, self.n_bnd_total,
                                      self.loss, self.dW)
        dist.all_reduce(self.dW, group=self.group)
        dist.all_reduce(self.loss, group=self.group)
        capi.adam_step(self.h, W, self.dW, lr, b1, b2, eps, t)
        return self.loss
