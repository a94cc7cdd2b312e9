"""Data parallelism over ranks (one process per GPU, torch.distributed).

The configurations of a batch are independent (Sec. 1: each proposal is one
prior sample pushed through the flow), so a global batch of B configurations
is split into contiguous ranges, one per rank: rank r takes configurations
[offset_r, offset_r + count_r) of the global batch, i.e. prior counters
counter0 + offset_r ... on its own GPU.  The union over ranks is exactly the
single-process batch, so results do not depend on the number of ranks.

Two exchange steps exist, both small:

- training (Sec. 1, shifted reverse KL; Sec. 3, Adam): the loss is the mean
  over the B configurations, so the global gradient is
  sum_r (count_r / B) * g_r with g_r the mean-loss gradient of rank r's
  range; one all-reduce of n_params FP32 values per step (974 KB for the 2D
  L=32, 24-coupling, hidden-32 flow), then every rank applies the same Adam
  update to its copy of the weights, which therefore stay identical;
- one global MH chain (Sec. 1, MH test with the Jacobian): the log-weights
  of all ranks gathered to one rank in global proposal order (8 B per
  proposal), where the serial accept/reject scan runs.  Independent chains
  per rank need no exchange at all.

The collectives are plain torch.distributed calls (NCCL on GPUs, gloo on the
CPU); no multicast or peer memory is used.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def partition(B: int, world: int, rank: int) -> tuple[int, int]:
    """(offset, count) of rank `rank`'s share of B configurations: the first
    B % world ranks take one extra configuration."""
    if world < 1 or not 0 <= rank < world or B < 0:
        raise ValueError("bad partition request")
    base, extra = divmod(B, world)
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def _rank_world(group):
    if not dist.is_available() or not dist.is_initialized():
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def allreduce_batch_mean(value: torch.Tensor, count: int, B: int, group=None) -> torch.Tensor:
    """In place: value <- sum over ranks of (count_r / B) * value_r, the mean
    over the global batch of per-rank means (a loss or its gradient)."""
    value.mul_(count / B)
    _, world = _rank_world(group)
    if world > 1:
        dist.all_reduce(value, op=dist.ReduceOp.SUM, group=group)
    return value


def dp_step(grad_fn, apply_fn, B: int, counter0: int, group=None):
    """One data-parallel training step, independent of how gradients are made.

    grad_fn(count, counter0) -> (loss, grad): mean loss (1-element tensor) and
    its gradient over `count` configurations whose prior counters start at
    `counter0`; apply_fn(grad) applies the optimiser update with the global
    gradient.  Returns the global mean loss.  Every rank must call it with
    the same B and counter0."""
    rank, world = _rank_world(group)
    off, n = partition(B, world, rank)
    if n == 0:
        raise ValueError("more ranks than configurations")
    loss, grad = grad_fn(n, counter0 + off)
    loss = allreduce_batch_mean(loss.clone(), n, B, group)
    allreduce_batch_mean(grad, n, B, group)
    apply_fn(grad)
    return loss


def dp_train_step(flow, phi4, B: int, seed: int, counter0: int, lr: float, adam_m, adam_v, adam_t: int,
                  workspace=None, group=None, beta1=0.9, beta2=0.999, adam_eps=1e-8):
    """dp_step on the GPU library: gf_flow_train_step (lr = 0, gradient out)
    over this rank's configurations, the all-reduce, then gf_flow_adam_step."""
    def grad_fn(n, c0):
        return flow.train_step(n, phi4, seed=seed, counter0=c0, lr=0.0, grad=True, workspace=workspace)

    def apply_fn(g):
        flow.adam_step(g, lr, adam_m, adam_v, adam_t, beta1=beta1, beta2=beta2, adam_eps=adam_eps)

    return dp_step(grad_fn, apply_fn, B, counter0, group)


def gather_logw(logw_local: torch.Tensor, B: int, dst: int = 0, group=None):
    """Gathers every rank's log-weights (its `partition` range of B proposals)
    to rank `dst` in global proposal order; returns the [B] tensor on `dst`,
    None elsewhere."""
    rank, world = _rank_world(group)
    if world == 1:
        return logw_local
    counts = [partition(B, world, r)[1] for r in range(world)]
    if logw_local.numel() != counts[rank]:
        raise ValueError("local log-weights do not match this rank's partition")
    width = max(counts)
    buf = torch.zeros(width, dtype=logw_local.dtype, device=logw_local.device)
    buf[:counts[rank]] = logw_local
    parts = [torch.empty_like(buf) for _ in range(world)] if rank == dst else None
    dist.gather(buf, parts, dst=dst, group=group)
    if rank != dst:
        return None
    return torch.cat([p[:c] for p, c in zip(parts, counts)])
