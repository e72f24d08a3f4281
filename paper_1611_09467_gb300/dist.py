"""The one exchange step of a multi-GPU gradient step (argument plumbing).

Configurations (Markov chains) are independent, so ranks shard them and
evaluate with no communication.  The estimator of Sec. II,
dE/dA = 2<Delta E> - 2<Delta><E>, is built from sums over configurations:
each rank forms its sums (sum E, count, sum E^2, sum Delta, sum E Delta) on
its GPU, one allreduce adds them across ranks, and each rank forms the means
of the whole job from the added sums on its GPU.  Every rank then holds the
same energy and gradient, as a single GPU would for the concatenated batch.
"""
from __future__ import annotations


def allreduce_sums(sums, group=None):
    """Adds a rank's gradient sums (a float64 tensor, NCCL on the GPU or gloo
    on the CPU) over the ranks of `group`, in place; a no-op on one rank."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    return sums


def distributed_gradient(peps, S, group=None):
    """Energy per site and gradient over every rank's configurations: local
    sums on this rank's GPU, one allreduce, the means on this rank's GPU."""
    sums = peps.gradient_sums(S)
    allreduce_sums(sums, group)
    return peps.gradient_from_sums(sums)
