"""FP64 CPU oracle of the placement loop around the density energy (arXiv 2307.12041,
Sec. IV: min_v f(v) = W_LSE(v) + lambda N(v), one Nesterov step per iteration, a
penalty update, and an overflow stop, all "as in ePlace", whose parameters the
paper does not restate).

TEST INFRASTRUCTURE ONLY: only the tests may import this module; it shares no code
with the CUDA library.

Definitions (pins at the block centres; a net e is a set of blocks):

* log-sum-exp wirelength with smoothing gamma, per net and axis
      W_e = gamma ln sum_{i in e} exp(x_i / gamma) + gamma ln sum_{i in e} exp(-x_i / gamma),
  summed over nets and both axes; it bounds the half-perimeter wirelength (HPWL)
  from above by at most 2 gamma ln |e| per net and axis and tends to it as gamma -> 0.
  Its gradient: dW_e/dx_i = softmax_e(x / gamma)_i - softmax_e(-x / gamma)_i.
* HPWL = sum_e (max - min of x over e) + (max - min of y over e).
* overflow on an m x m grid of bins: with D_b the total block area inside bin b
  (exact overlap areas) and A_b the bin area,
      tau = sum_b max(D_b - rho_t A_b, 0) / (total area of the movable blocks).
* one Nesterov step (accelerated gradient with momentum coefficient from the
  sequence a_{k+1} = (1 + sqrt(4 a_k^2 + 1)) / 2):
      u_{k+1} = clamp(v_k - alpha_k g_k),
      v_{k+1} = clamp(u_{k+1} + (a_k - 1) / a_{k+1} (u_{k+1} - u_k)),
  clamp keeping each block inside the die (centre in [w/2, W - w/2]); fixed blocks
  do not move.
"""
from __future__ import annotations

import math

import numpy as np


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def lse_wirelength(x, y, net_ptr, net_pin, gamma):
    """(W_LSE, HPWL, dW/dx, dW/dy) in FP64; net e's pins are net_pin[net_ptr[e]:net_ptr[e+1]]."""
    x, y = _f64(x), _f64(y)
    gx = np.zeros_like(x)
    gy = np.zeros_like(y)
    W = 0.0
    hp = 0.0
    for e in range(len(net_ptr) - 1):
        pins = np.asarray(net_pin[net_ptr[e]:net_ptr[e + 1]])
        if len(pins) < 2:
            continue
        for coord, g in ((x, gx), (y, gy)):
            v = coord[pins]
            hi, lo = v.max(), v.min()
            ep = np.exp((v - hi) / gamma)          # shifted: the largest term is 1
            en = np.exp((lo - v) / gamma)
            W += hi + gamma * math.log(ep.sum()) - lo + gamma * math.log(en.sum())
            hp += hi - lo
            np.add.at(g, pins, ep / ep.sum() - en / en.sum())
    return W, hp, gx, gy


def hpwl(x, y, net_ptr, net_pin):
    return lse_wirelength(x, y, net_ptr, net_pin, 1.0)[1]


def overflow(x, y, w, h, movable, W, H, m, target=1.0):
    """tau on an m x m grid from the exact overlap area of every block with every bin."""
    x, y, w, h = _f64(x), _f64(y), _f64(w), _f64(h)
    wb, hb = W / m, H / m
    D = np.zeros((m, m))
    for i in range(len(x)):
        x0, x1 = x[i] - w[i] / 2, x[i] + w[i] / 2
        y0, y1 = y[i] - h[i] / 2, y[i] + h[i] / 2
        l0, l1 = max(0, int(math.floor(x0 / wb))), min(m - 1, int(math.floor(x1 / wb)))
        j0, j1 = max(0, int(math.floor(y0 / hb))), min(m - 1, int(math.floor(y1 / hb)))
        for l in range(l0, l1 + 1):
            ox = min(x1, (l + 1) * wb) - max(x0, l * wb)
            if ox <= 0:
                continue
            for j in range(j0, j1 + 1):
                oy = min(y1, (j + 1) * hb) - max(y0, j * hb)
                if oy > 0:
                    D[l, j] += ox * oy
    mov = np.ones(len(x), bool) if movable is None else np.asarray(movable, bool)
    area = float(np.sum(w[mov] * h[mov]))
    return float(np.maximum(D - target * wb * hb, 0.0).sum() / area), D


def nesterov_next_a(a):
    return (1.0 + math.sqrt(4.0 * a * a + 1.0)) / 2.0


def nesterov_step(u, v, g, w, L, alpha, a, movable=None):
    """One coordinate's update (x with widths w and die size L, or y with h, H):
    returns (u_next, v_next)."""
    u, v, g, w = _f64(u), _f64(v), _f64(g), _f64(w)
    lo, hi = w / 2, L - w / 2
    un = np.clip(v - alpha * g, lo, hi)
    an = nesterov_next_a(a)
    vn = np.clip(un + (a - 1.0) / an * (un - u), lo, hi)
    if movable is not None:                 # fixed blocks keep both solutions: they do not move
        mov = np.asarray(movable, bool)
        un = np.where(mov, un, u)
        vn = np.where(mov, vn, v)
    return un, vn
