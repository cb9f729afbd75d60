"""Seeded synthetic placements.

This module only draws inputs (block centres, sizes, charges and the descent
jitter).  It holds none of the series arithmetic, so the FP64 oracle and the
CUDA path can both be fed from it without sharing any of the method's code.

The paper evaluates on the ISPD 2005/2006 contest placements (Sec. V), which
are not available here; the workloads below stand in for them with seeded
distributions of the same character: a die of 1 x 1, millions of small
standard cells of one row height, a small fraction of macros, and clustered
centres.

Every array is float32 (the library's input type).  The die is [0, W] x [0, H].
Centres are clamped so that each block lies inside the die, which is the
setting of Eq. (global density): theta_i is supported inside R.  The one
exception is `out_of_die_blocks`, which draws blocks that overhang an edge, lie
outside the die or are wider than it, for the edge-case tests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 2307_12041


@dataclass
class Placement:
    """A set of rectangular blocks on a die, plus the mode counts to use."""
    W: float
    H: float
    x: np.ndarray
    y: np.ndarray
    w: np.ndarray
    h: np.ndarray
    c: np.ndarray | None
    Mx: int
    My: int
    movable: np.ndarray | None = None   # bool mask; None = all movable
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def subset(self, idx) -> "Placement":
        idx = np.asarray(idx)
        return Placement(self.W, self.H, self.x[idx].copy(), self.y[idx].copy(),
                         self.w[idx].copy(), self.h[idx].copy(),
                         None if self.c is None else self.c[idx].copy(),
                         self.Mx, self.My,
                         None if self.movable is None else self.movable[idx].copy(),
                         self.name + "[subset]", dict(self.meta))


def _streams(seed: int, k: int):
    ss = np.random.SeedSequence(seed)
    return [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(k)]


def lognormal_with_mean(rng, mean: float, sigma: float, size: int) -> np.ndarray:
    """Lognormal whose ARITHMETIC mean is `mean` and log-space std is sigma:
    mu = ln(mean) - sigma^2 / 2."""
    mu = math.log(mean) - 0.5 * sigma * sigma
    return rng.lognormal(mu, sigma, size)


def _clamp_centres(x, w, L):
    lo = 0.5 * w
    hi = L - 0.5 * w
    return np.minimum(np.maximum(x, lo), hi)


def uniform_blocks(n: int, Mx: int, My: int, seed: int, W: float = 1.0, H: float = 1.0,
                   mean_size: float = 0.004, sigma: float = 0.5, charge: bool = False,
                   name: str = "uniform") -> Placement:
    """Centres uniform in the die, w and h lognormal (given arithmetic mean)."""
    r_w, r_h, r_x, r_y, r_c = _streams(seed, 5)
    w = lognormal_with_mean(r_w, mean_size * W, sigma, n)
    h = lognormal_with_mean(r_h, mean_size * H, sigma, n)
    w = np.minimum(w, W)
    h = np.minimum(h, H)
    x = 0.5 * w + r_x.random(n) * (W - w)
    y = 0.5 * h + r_y.random(n) * (H - h)
    c = r_c.uniform(0.5, 1.5, n) if charge else None
    return Placement(W, H, x.astype(np.float32), y.astype(np.float32),
                     w.astype(np.float32), h.astype(np.float32),
                     None if c is None else c.astype(np.float32), Mx, My, name=name)


def cell_mix(n: int, Mx: int, My: int, seed: int, W: float = 1.0, H: float = 1.0,
             n_clusters: int = 20, cluster_sigma: float = 0.1, macro_frac: float = 0.01,
             name: str = "cell-mix") -> Placement:
    """Standard cells (h = 0.001 H, w lognormal with mean 0.002 W, sigma 0.5) plus a
    fraction of macros (w, h uniform in [0.01, 0.05] of the die); centres drawn from
    an equal-weight mixture of Gaussians (means uniform in [0.1, 0.9]^2, std 0.1),
    then clamped into the die."""
    r_kind, r_w, r_mw, r_mh, r_comp, r_mu, r_x, r_y = _streams(seed, 8)
    is_macro = r_kind.random(n) < macro_frac
    w = lognormal_with_mean(r_w, 0.002 * W, 0.5, n)
    h = np.full(n, 0.001 * H)
    nm = int(is_macro.sum())
    w[is_macro] = r_mw.uniform(0.01, 0.05, nm) * W
    h[is_macro] = r_mh.uniform(0.01, 0.05, nm) * H
    w = np.minimum(w, W)
    means = r_mu.uniform(0.1, 0.9, (n_clusters, 2))
    comp = r_comp.integers(0, n_clusters, n)
    x = means[comp, 0] * W + r_x.normal(0.0, cluster_sigma, n) * W
    y = means[comp, 1] * H + r_y.normal(0.0, cluster_sigma, n) * H
    x = _clamp_centres(x, w, W)
    y = _clamp_centres(y, h, H)
    return Placement(W, H, x.astype(np.float32), y.astype(np.float32),
                     w.astype(np.float32), h.astype(np.float32), None, Mx, My,
                     name=name, meta={"macros": nm})


def cells_plus_fixed_macros(n_cells: int, n_macros: int, Mx: int, My: int, seed: int,
                            W: float = 1.0, H: float = 1.0) -> Placement:
    """`cell_mix` cells followed by fixed macros (w, h uniform in [0.02, 0.08] of the
    die, centres uniform); the macros are flagged not movable."""
    p = cell_mix(n_cells, Mx, My, seed, W, H, name="cells+fixed-macros")
    r_w, r_h, r_x, r_y = _streams(seed + 7919, 4)
    mw = r_w.uniform(0.02, 0.08, n_macros) * W
    mh = r_h.uniform(0.02, 0.08, n_macros) * H
    mx = 0.5 * mw + r_x.random(n_macros) * (W - mw)
    my = 0.5 * mh + r_y.random(n_macros) * (H - mh)
    cat = lambda a, b: np.concatenate([a, b.astype(np.float32)])
    mov = np.concatenate([np.ones(n_cells, bool), np.zeros(n_macros, bool)])
    return Placement(W, H, cat(p.x, mx), cat(p.y, my), cat(p.w, mw), cat(p.h, mh),
                     None, Mx, My, movable=mov, name=p.name,
                     meta={"cells": n_cells, "fixed_macros": n_macros})


OUT_OF_DIE_KINDS = ("inside", "overhang", "centre-outside", "wider-than-die", "negative", "far")


def out_of_die_blocks(n: int, Mx: int, My: int, seed: int, W: float = 1.0, H: float = 1.0,
                      charge: bool = True) -> Placement:
    """Blocks the workload generators never make: the die R = [0, W] x [0, H] of
    Eq. (global density) no longer contains every block.  Per axis, each block is
    drawn from one of OUT_OF_DIE_KINDS (cyclically, so every kind occurs on both
    axes and in combination):
      inside          centre uniform with the block inside, size lognormal (mean 0.05)
      overhang        the block straddles a die edge (left/bottom or right/top)
      centre-outside  the centre lies up to half a size beyond an edge
      wider-than-die  size 1 to 2.5 times the die, centre uniform in the die
      negative        centre in [-1.5 L, 0): the block mostly or wholly below 0
      far             centre in (L, 3 L]: beyond the far edge, past 2 L
    Charges uniform in [0.5, 1.5] (or None)."""
    r_kx, r_ky, r_sx, r_sy, r_px, r_py, r_side, r_c = _streams(seed, 8)
    kx = (np.arange(n) + r_kx.integers(0, len(OUT_OF_DIE_KINDS))) % len(OUT_OF_DIE_KINDS)
    ky = (np.arange(n) // len(OUT_OF_DIE_KINDS) + r_ky.integers(0, len(OUT_OF_DIE_KINDS))) \
        % len(OUT_OF_DIE_KINDS)

    def axis(kind, r_s, r_p, L):
        size = lognormal_with_mean(r_s, 0.05 * L, 0.5, n)
        u = r_p.random(n)
        side = r_side.random(n) < 0.5
        pos = 0.5 * size + u * (L - size)                                # inside
        edge = np.where(side, 0.0, L)
        sgn = np.where(side, 1.0, -1.0)
        over = edge + sgn * (u - 0.5) * size                             # straddles the edge
        beyond = edge - sgn * u * 0.5 * size                             # centre past the edge
        wide = r_s.uniform(1.0, 2.5, n) * L
        pos = np.where(kind == 1, over, pos)
        pos = np.where(kind == 2, beyond, pos)
        size = np.where(kind == 3, wide, size)
        pos = np.where(kind == 3, u * L, pos)
        pos = np.where(kind == 4, -1.5 * L * u, pos)
        pos = np.where(kind == 5, L + 2.0 * L * (1.0 - u), pos)
        return pos, size

    x, w = axis(kx, r_sx, r_px, W)
    y, h = axis(ky, r_sy, r_py, H)
    c = r_c.uniform(0.5, 1.5, n) if charge else None
    return Placement(W, H, x.astype(np.float32), y.astype(np.float32), w.astype(np.float32),
                     h.astype(np.float32), None if c is None else c.astype(np.float32), Mx, My,
                     name="out-of-die", meta={"kinds_x": kx, "kinds_y": ky})


# The five workloads: (n, Mx, My, recipe).  Index 0 is the small case the oracle
# finishes in seconds; index 1 is the throughput workload.
WORKLOADS = {
    0: dict(name="uniform-2k-64x64", n=2_000, Mx=64, My=64, kind="uniform"),
    1: dict(name="cellmix-200k-512x512", n=200_000, Mx=512, My=512, kind="mix"),
    2: dict(name="cellmix-1M-1024x1024", n=1_000_000, Mx=1024, My=1024, kind="mix"),
    3: dict(name="cells2M+500fixed-1024x1024", n=2_000_000, Mx=1024, My=1024, kind="fixed",
            n_macros=500),
    4: dict(name="cellmix-10M-2048x2048", n=10_000_000, Mx=2048, My=2048, kind="mix"),
}


def workload(index: int, n: int | None = None) -> Placement:
    """Draw workload `index` (0..4) with seed BASE_SEED + index.  `n` overrides the
    block count (same recipe, same seed) for scaled-down runs."""
    spec = WORKLOADS[index]
    seed = BASE_SEED + index
    nn = spec["n"] if n is None else int(n)
    if spec["kind"] == "uniform":
        p = uniform_blocks(nn, spec["Mx"], spec["My"], seed, name=spec["name"])
    elif spec["kind"] == "mix":
        p = cell_mix(nn, spec["Mx"], spec["My"], seed, name=spec["name"])
    else:
        p = cells_plus_fixed_macros(nn, spec["n_macros"], spec["Mx"], spec["My"], seed)
        p.name = spec["name"]
    return p



# ---- placement-loop inputs (Sec. IV) --------------------------------------------
# The ISPD netlists are not available; the stand-in is a netlist with the usual
# character: about one net per cell, mostly two- and three-pin nets with a tail up
# to 16 pins, and locality (a net's pins lie close together in a hidden target
# layout), on standard cells of one row height at a set utilisation, started from
# a dense cluster at the die centre so that the loop has to spread them.

NET_DEGREES = np.array([2, 3, 4, 5, 6, 8, 12, 16])
NET_DEGREE_P = np.array([0.55, 0.18, 0.1, 0.06, 0.04, 0.03, 0.02, 0.02])


def placement_cells(n: int, M: int, seed: int, util: float = 0.7, W: float = 1.0, H: float = 1.0,
                    start_sigma: float = 0.05) -> Placement:
    """n standard cells (h one row, w lognormal with sigma 0.5) scaled so that their
    total area is util * W * H; centres normal around the die centre (std
    start_sigma of the die), clamped.  M modes per axis."""
    r_w, r_x, r_y = _streams(seed, 3)
    row = 0.001 * H
    w = lognormal_with_mean(r_w, 0.002 * W, 0.5, n)
    h = np.full(n, row)
    w *= util * W * H / float(np.sum(w * h))
    w = np.minimum(w, W)
    x = _clamp_centres(0.5 * W + r_x.normal(0.0, start_sigma, n) * W, w, W)
    y = _clamp_centres(0.5 * H + r_y.normal(0.0, start_sigma, n) * H, h, H)
    return Placement(W, H, x.astype(np.float32), y.astype(np.float32), w.astype(np.float32),
                     h.astype(np.float32), None, M, M, name=f"place-{n}-{M}x{M}",
                     meta={"util": util, "start_sigma": start_sigma})


def netlist(n_cells: int, seed: int, nets_per_cell: float = 1.0, window: int = 64):
    """(net_ptr, net_pin) int64: net degrees from NET_DEGREES / NET_DEGREE_P; a net's
    pins are distinct cells within `window` positions of a random start in a hidden
    order (the cells sorted along a space-filling curve of a random target layout),
    so that nets are local.  Every cell gets at least one net (two-pin nets to a
    neighbour in the order are added for cells left out)."""
    r_ord, r_deg, r_start, r_pick = _streams(seed, 4)
    # hidden target layout: random points in a 1024 x 1024 grid, ordered by a Morton curve
    g = r_ord.integers(0, 1024, (n_cells, 2))
    def spread(v):
        v = v.astype(np.int64)
        out = np.zeros_like(v)
        for b in range(10):
            out |= ((v >> b) & 1) << (2 * b)
        return out
    order = np.argsort(spread(g[:, 0]) | (spread(g[:, 1]) << 1), kind="stable")
    n_nets = max(1, int(round(nets_per_cell * n_cells)))
    deg = r_deg.choice(NET_DEGREES, n_nets, p=NET_DEGREE_P)
    deg = np.minimum(deg, max(2, n_cells))
    start = r_start.integers(0, max(1, n_cells - window), n_nets)
    pins = []
    for d, s0 in zip(deg, start):
        span = min(window, n_cells)
        pick = r_pick.choice(span, d, replace=False)
        pins.append(order[np.minimum(s0 + pick, n_cells - 1)])
    used = np.zeros(n_cells, bool)
    for pp in pins:
        used[pp] = True
    rank = np.empty(n_cells, np.int64)
    rank[order] = np.arange(n_cells)
    for c in np.flatnonzero(~used):                 # a two-pin net to the next cell in the order
        k = rank[c]
        other = order[k + 1] if k + 1 < n_cells else order[k - 1]
        pins.append(np.array([c, other]))
    ptr = np.concatenate([[0], np.cumsum([len(pp) for pp in pins])]).astype(np.int64)
    return ptr, np.concatenate(pins).astype(np.int64)
