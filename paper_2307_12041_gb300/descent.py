"""Gradient-descent driver over block positions (a stand-in for the placer loop of
Sec. IV, whose Nesterov parameters the paper does not restate).

Each step evaluates E and its gradient through the C ABI, then moves the
movable blocks:  x <- clamp(x - lr * dE/dx + j, w/2, W - w/2)  (same for y), with
a seed-fixed jitter j ~ N(0, (jitter * W)^2) per block and step drawn on the host
(PCG64 keyed by (seed, step)) and uploaded.

Chunked evaluation.  The coefficients are a sum over blocks (Eq. aup sums over
i), so with the blocks cut into chunks, a = sum_c a(chunk c) (pp_coeffs per chunk)
and each chunk's energies and gradients follow from pp_grad with that total a.
This bounds the workspace by the chunk size for placements too large for one
call.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np
import torch

from . import binding, synth


@dataclass
class DescentResult:
    energy: List[float] = field(default_factory=list)
    x: Optional[torch.Tensor] = None
    y: Optional[torch.Tensor] = None
    ms_per_step: float = 0.0


def evaluate_chunked(x, y, w, h, c, W, H, Mx, My, prec="tf32", chunk: Optional[int] = None):
    """(gx, gy, E) of the whole placement; with `chunk`, the blocks are processed
    in chunks of that many blocks (coefficients summed over chunks first)."""
    n = x.numel()
    if not chunk or chunk >= n:
        gx, gy, _, et = binding.grad(x, y, w, h, c, W, H, Mx, My, prec)
        return gx, gy, et
    cuts = list(range(0, n, chunk)) + [n]
    sl = lambda t, a, b: None if t is None else t[a:b]
    a = None
    for s, e in zip(cuts[:-1], cuts[1:]):
        ac = binding.coeffs(x[s:e], y[s:e], w[s:e], h[s:e], sl(c, s, e), W, H, Mx, My, prec)
        a = ac if a is None else a + ac
    gx = torch.empty_like(x)
    gy = torch.empty_like(y)
    E = torch.zeros(1, dtype=torch.float64, device=x.device)
    for s, e in zip(cuts[:-1], cuts[1:]):
        gxc, gyc, _, ec = binding.grad(x[s:e], y[s:e], w[s:e], h[s:e], sl(c, s, e), W, H, Mx, My,
                                       prec, a=a)
        gx[s:e] = gxc
        gy[s:e] = gyc
        E += ec
    return gx, gy, E


def descend(p: synth.Placement, steps: int, lr: float = 1e-4, jitter: float = 1e-6,
            seed: int = synth.BASE_SEED, prec: str = "tf32", chunk: Optional[int] = None,
            device="cuda", callback: Optional[Callable] = None) -> DescentResult:
    """Run `steps` descent steps on placement `p`; callback(k, x, y, gx, gy, E)
    is called after each evaluation (before the move)."""
    dev = torch.device(device)
    x, y, w, h, c = binding.to_device(p, dev)
    x = x.clone()
    y = y.clone()
    mov = None if p.movable is None else torch.from_numpy(p.movable).to(dev)
    lo_x, hi_x = 0.5 * w, p.W - 0.5 * w
    lo_y, hi_y = 0.5 * h, p.H - 0.5 * h
    res = DescentResult()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for k in range(steps):
        gx, gy, E = evaluate_chunked(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec, chunk)
        res.energy.append(E)
        if callback is not None:
            callback(k, x, y, gx, gy, E)
        j = torch.from_numpy(synth.descent_jitter(p.n, k, seed, jitter * p.W)).to(dev)
        dx = -lr * gx + j[0]
        dy = -lr * gy + j[1]
        if mov is not None:
            dx = torch.where(mov, dx, torch.zeros_like(dx))
            dy = torch.where(mov, dy, torch.zeros_like(dy))
        x = torch.minimum(torch.maximum(x + dx, lo_x), hi_x)
        y = torch.minimum(torch.maximum(y + dy, lo_y), hi_y)
    t1.record()
    torch.cuda.synchronize()
    binding.sync_status(dev)
    res.energy = [float(e.item()) for e in res.energy]
    res.x, res.y = x, y
    res.ms_per_step = t0.elapsed_time(t1) / max(steps, 1)
    return res
