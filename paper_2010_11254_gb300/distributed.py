"""One tree's evaluation split across processes, one GPU each.

Every process builds the same tree from the same particles (the build is
cheap next to the evaluation) and evaluates a contiguous share of the groups
of the active set, Morton-ordered (sfg_set_group_share); each group is
evaluated by exactly one process.  Forward rows of other shares come out as
zeros and the adjoint's gradients are this share's part of the sums, so one
all-reduce (sum) of every output assembles the unsplit result.  The paper's
runs split the tree work over MPI ranks by domain decomposition (STARFORGE
methods paper, Sec. 2.2); here the split is over groups of targets.

Collectives go through torch.distributed on the caller's process group
(NCCL between GPUs); the data path has no other exchange.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def group_share(n_groups: int, rank: int, world: int) -> tuple[int, int]:
    """The groups [g0, g1) of share `rank` of `world` (the library's rule)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return n_groups * rank // world, n_groups * (rank + 1) // world


def combine(*tensors: torch.Tensor, group=None) -> None:
    """Sum every tensor over the processes of `group`, in place."""
    for t in tensors:
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)


def scatter_rows(t: torch.Tensor, group=None) -> torch.Tensor:
    """Sum `t` (first axis: particles) over the processes of `group` and keep
    this process's contiguous block of rows (a reduce-scatter: ceil(n / world)
    rows per process, the last block shorter)."""
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    n = t.shape[0]
    per = -(-n // world)
    pad = per * world - n
    src = torch.cat([t, t.new_zeros((pad,) + tuple(t.shape[1:]))]) if pad else t.contiguous()
    out = t.new_empty((per,) + tuple(t.shape[1:]))
    if dist.get_backend(group) == "nccl":
        dist.reduce_scatter_tensor(out, src, op=dist.ReduceOp.SUM, group=group)
    else:  # backends without a reduce-scatter: all-reduce, then keep the block
        dist.all_reduce(src, op=dist.ReduceOp.SUM, group=group)
        out.copy_(src[rank * per:(rank + 1) * per])
    return out[:max(0, min(per, n - rank * per))]


def accel(tree, active=None, group=None):
    """(accel, phi) of every active row, this process evaluating its share of
    the groups; the rows of all shares are assembled by one all-reduce."""
    tree.set_group_share(dist.get_rank(group), dist.get_world_size(group))
    acc, phi = tree.accel(active)
    combine(acc, phi, group=group)
    return acc, phi


def accel_vjp(tree, active, cot_a, cot_phi=None, group=None, scatter: bool = False):
    """(d_pos, d_mass) of the split adjoint: this process's share of the
    groups, summed over processes by one all-reduce, or with scatter=True one
    reduce-scatter that leaves each process its block of particles."""
    tree.set_group_share(dist.get_rank(group), dist.get_world_size(group))
    d_pos, d_mass = tree.accel_vjp(active, cot_a, cot_phi)
    if scatter:
        return scatter_rows(d_pos, group), scatter_rows(d_mass, group)
    combine(d_pos, d_mass, group=group)
    return d_pos, d_mass
