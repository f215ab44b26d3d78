"""View-sharded texture-fitting step over several GPUs (one process each).

The fitting step of the paper (Sec. 3 "Texturing Meshes": the textures are
optimised against a photometric loss summed over training views) is a sum of
independent per-view terms.  So N ranks each render and differentiate their
own share of the views, and the FP32 texel gradients of the step are the sum
of the ranks' partial gradients: ONE all-reduce (sum) per step, issued after
the rank's fused forward + adjoint and before the caller's optimizer step.
Nothing else is exchanged: no peer memory is handed to any kernel, and the
all-reduce is torch.distributed's (NCCL between GPUs, gloo between CPU ranks).

Partition: views are dealt round-robin, rank r owns views r, r + N, r + 2N,
... of the step's view list.
"""

from __future__ import annotations

from typing import Callable, List, Optional, Sequence

import torch


def view_shard(n_views: int, rank: int, world: int) -> List[int]:
    """Indices of the views rank `rank` of `world` renders: rank, rank + world, ..."""
    if world < 1 or not 0 <= rank < world or n_views < 0:
        raise ValueError(f"bad shard request: {n_views} views, rank {rank} of {world}")
    return list(range(rank, n_views, world))


class ShardedFittingStep:
    """One fitting step over a view set split across the ranks of a process
    group.

    grads          this rank's FP32 texel-gradient tensors (one per shell);
                   after a step they hold the gradient over ALL views, equal
                   on every rank
    compute_grads  callable(views) that ADDS the gradient of the rank's views
                   into `grads` (on the GPU: one vs_render_batch over those
                   views with do_backward=1; on CPU ranks: any adjoint, e.g.
                   the oracle's in the tests)
    n_views        size of the step's view list
    zero_grads     zero `grads` before the rank's work (the step's gradient
                   alone, not accumulated over steps)
    The rank and world size come from torch.distributed when it is
    initialised (group = None: the default group), else 0 of 1, in which
    case no collective runs.
    """

    def __init__(self, grads: Sequence[torch.Tensor], compute_grads: Callable[[List[int]], None], n_views: int,
                 rank: Optional[int] = None, world: Optional[int] = None, group=None, zero_grads: bool = True):
        import torch.distributed as dist
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        if world is None:
            world = self.dist.get_world_size(group) if self.dist else 1
        if rank is None:
            rank = self.dist.get_rank(group) if self.dist else 0
        if world > 1 and self.dist is None:
            raise RuntimeError("a sharded step over several ranks needs torch.distributed initialised")
        for g in grads:
            if g.dtype != torch.float32 or not g.is_contiguous():
                raise ValueError("texel gradients must be contiguous float32 tensors")
        self.grads = list(grads)
        self.compute_grads = compute_grads
        self.rank, self.world, self.group = rank, world, group
        self.views = view_shard(n_views, rank, world)
        self.zero_grads = zero_grads

    def __call__(self) -> List[torch.Tensor]:
        if self.zero_grads:
            for g in self.grads:
                g.zero_()
        self.compute_grads(self.views)
        if self.world > 1:
            # one sum over the ranks per gradient tensor, all in flight at once
            work = [self.dist.all_reduce(g, op=self.dist.ReduceOp.SUM, group=self.group, async_op=True)
                    for g in self.grads]
            for w in work:
                w.wait()
        return self.grads
