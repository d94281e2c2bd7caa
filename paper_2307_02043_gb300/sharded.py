"""Illumination sharding of the mini-batch gradient over several GPUs (one
process per GPU, torch.distributed for the one collective).

Eq. 4.1: grad F_s = (S/L) sum_{l in S_s} grad f_l is a plain sum over the
illuminations of the subset, so each rank computes the partial sum over its
share of S_s (interleaved: rank r takes S_s[r], S_s[r + world], ...) and one
all-reduce (sum) of the N gradient values, plus one of the loss, gives every
rank grad F_s and F_s.  The SR1 update, the quasi-Newton point and the
weighted proximal mapping then run replicated on every rank: they are
deterministic and every rank holds the same x, so the replicas stay
identical and no other exchange is needed.  A rank keeps the stored forward
fields (warm start) of its own illuminations only, which is consistent
because a subset is always split the same way.

Every numerical step still runs in libmqnpm; this module only splits the
illumination list and sums the partial results.
"""
from __future__ import annotations

from typing import Callable, List, Sequence, Tuple

import torch
import torch.distributed as dist


def shard(illum: Sequence[int], rank: int, world: int) -> List[int]:
    """Rank `rank`'s share of an illumination list (interleaved, sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    return [int(l) for l in list(illum)[rank::world]]


def sharded_gradient(grad_fn: Callable[[List[int], float], Tuple[torch.Tensor, float]], illum: Sequence[int],
                     scale: float, rank: int, world: int, zeros: Callable[[], torch.Tensor],
                     all_reduce=None) -> Tuple[torch.Tensor, float]:
    """scale * sum_{l in illum} (grad f_l, f_l) on every rank: grad_fn(share,
    scale) -> (gradient tensor, loss) gives this rank's partial sum; a rank
    with an empty share contributes zeros() and 0; all_reduce(t) sums a tensor
    over the ranks in place (torch.distributed.all_reduce when None)."""
    mine = shard(illum, rank, world)
    if mine:
        g, loss = grad_fn(mine, scale)
    else:
        g, loss = zeros(), 0.0
    if world == 1:
        return g, float(loss)
    reduce = all_reduce if all_reduce is not None else dist.all_reduce
    reduce(g)
    lt = torch.tensor([float(loss)], dtype=torch.float64, device=g.device)
    reduce(lt)
    return g, float(lt.item())


class ShardedStep:
    """One iteration of Algorithm 4.1 on a libmqnpm handle with the subset
    gradient sharded over the ranks of the default process group (or of no
    group: world = 1, where it computes exactly what handle.step does)."""

    def __init__(self, handle, rank: int = None, world: int = None):
        self.h = handle
        initialized = dist.is_available() and dist.is_initialized()
        self.rank = rank if rank is not None else (dist.get_rank() if initialized else 0)
        self.world = world if world is not None else (dist.get_world_size() if initialized else 1)
        self.scale = handle.S / handle.L

    def gradient(self, x: torch.Tensor, illum: Sequence[int]):
        h = self.h

        def grad_fn(mine, scale):
            g, loss, its = h.grad_batch(x, mine, scale, allow_not_converged=True)
            grad_fn.its = its
            return g, loss

        grad_fn.its = []
        g, loss = sharded_gradient(grad_fn, illum, self.scale, self.rank, self.world, lambda: torch.zeros_like(x))
        return g, loss, grad_fn.its

    def step(self, x: torch.Tensor) -> dict:
        subset, illum = self.h.step_subset()
        g, loss, its = self.gradient(x, illum)
        info = self.h.step_with_gradient(x, g, loss)
        info["illum_this_rank"] = len(shard(illum, self.rank, self.world))
        info["krylov_iters_this_rank"] = sum(a + b for a, b in its)
        return info
