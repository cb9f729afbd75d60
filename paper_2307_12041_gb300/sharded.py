"""One placement's blocks shared out over processes (one GPU each).

The coefficients are a sum over blocks (Eq. aup, au0, a0p sum over i), so with
the blocks partitioned across ranks the evaluation needs one exchange:

  1. each rank adds its own blocks' coefficients into an FP64 Mx x My array
     (pp_coeffs_accumulate), starting from zero;
  2. one all-reduce (sum) of that array over the ranks: Mx * My doubles;
  3. every rank rounds the sum to the float32 coefficients a (pp_coeffs_accumulate
     with no blocks), then evaluates its own blocks' N_i and gradient against the
     whole placement's a (pp_grad with a given), and the total energy
     E = 1/2 sum_uv a_uv S_uv from a (pp_energy_from_coeffs): the same value on
     every rank, so E needs no second collective.

The ranks' block ranges are contiguous and of equal size (block_range).  The
library calls are reached through an `ops` object so that the partition, the
collective and the row ownership can be exercised by CPU processes (gloo) with
stand-in arithmetic; `LibraryOps` is the only implementation the product uses.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import binding


def block_range(n: int, world: int, rank: int):
    """[start, stop) of rank's blocks: contiguous, sizes differing by at most one,
    in rank order, covering 0..n-1 exactly once."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    q, r = divmod(n, world)
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


class LibraryOps:
    """The CUDA library's entry points, as the sharded evaluation uses them."""

    @staticmethod
    def zeros64(Mx, My, device):
        return torch.zeros((Mx, My), dtype=torch.float64, device=device)

    @staticmethod
    def accumulate(x, y, w, h, c, W, H, Mx, My, a64, prec):
        binding.coeffs_accumulate(x, y, w, h, c, W, H, Mx, My, a64, prec)

    @staticmethod
    def round(a64, W, H, prec):
        Mx, My = a64.shape
        a = torch.empty((Mx, My), dtype=torch.float32, device=a64.device)
        e = torch.empty(0, dtype=torch.float32, device=a64.device)
        binding.coeffs_accumulate(e, e, e, e, None, W, H, Mx, My, a64, prec, a_out=a)
        return a

    @staticmethod
    def grad(x, y, w, h, c, W, H, Mx, My, prec, a):
        gx, gy, eb, _ = binding.grad(x, y, w, h, c, W, H, Mx, My, prec, a=a, want_energy=True)
        return gx, gy, eb

    @staticmethod
    def energy(a, W, H):
        return binding.energy_from_coeffs(a, W, H)


def evaluate(x, y, w, h, c, W, H, Mx, My, prec="tf32", group=None, ops=None):
    """Energy and gradient of a placement whose blocks are shared out over the ranks
    of `group` (torch.distributed; None = the default group, or a single process
    when torch.distributed is not initialised).  x, y, w, h, c hold THIS rank's
    blocks.  Returns (gx, gy, N_i) of this rank's blocks, E of the whole placement
    (1-element float64 tensor) and the whole placement's coefficients a."""
    import torch.distributed as dist
    ops = ops or LibraryOps
    a64 = ops.zeros64(Mx, My, x.device)
    ops.accumulate(x, y, w, h, c, W, H, Mx, My, a64, prec)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(a64, op=dist.ReduceOp.SUM, group=group)
    a = ops.round(a64, W, H, prec)
    gx, gy, eb = ops.grad(x, y, w, h, c, W, H, Mx, My, prec, a)
    return gx, gy, eb, ops.energy(a, W, H), a


def shard(p, world: int, rank: int):
    """This rank's part of a synth.Placement (its contiguous block range)."""
    import numpy as np
    s, e = block_range(p.n, world, rank)
    return p.subset(np.arange(s, e))
