"""Pins of the element-wise forward-error bound (tests/parity_bounds.py) on the CPU.

A TF32 or BF16x3 evaluation emulated in FP64 -- every operand rounded as the tensor
cores see it (TF32: 11 significant bits, nearest; BF16x3: hi + lo bf16 split with
the lo*lo product dropped) -- must lie inside the bound, and not far inside it
(the bound is not vacuous); plausible kernel mistakes (a dropped block, a flipped
mode, a shifted mode index, a gradient sign) must break it.
"""
import math

import numpy as np
import pytest

from oracle import series as O
from paper_2307_12041_gb300 import synth
from parity_bounds import bound_ratios


def rnd(x, bits):
    """Round to `bits` significant bits, nearest."""
    m, e = np.frexp(np.asarray(x, np.float64))
    return np.ldexp(np.round(np.ldexp(m, bits)), e - bits)


def op(x, prec):
    if prec == "tf32":
        return rnd(x, 11)
    hi = rnd(x, 8)
    return hi, rnd(x - hi, 8)


def mul_sum(A, B, prec):
    """A^T B (contraction over the first index) as the tensor cores form it."""
    if prec == "tf32":
        return op(A, prec).T @ op(B, prec)
    ah, al = op(A, prec)
    bh, bl = op(B, prec)
    return ah.T @ bh + ah.T @ bl + al.T @ bh


def emulate(p, prec):
    """Coefficients, N, gradient and E in the scaled form the kernels use."""
    W, H, Mx, My = float(p.W), float(p.H), p.Mx, p.My
    x, y, w, h = (np.asarray(v, np.float64) for v in (p.x, p.y, p.w, p.h))
    cc = np.ones(p.n) if p.c is None else np.asarray(p.c, np.float64)
    ku = np.arange(Mx) * math.pi / W
    lv = np.arange(My) * math.pi / H
    fu = 2.0 * W / (math.pi * np.maximum(np.arange(Mx), 1))
    gv = 2.0 * H / (math.pi * np.maximum(np.arange(My), 1))
    Ix, Jx = O.rect_integrals(x, w, W, Mx)
    Iy, Jy = O.rect_integrals(y, h, H, My)
    Xs = cc[:, None] * Ix / fu          # scaled basis, |values| <= |c|
    Ys = Iy / gv
    Xh = -cc[:, None] * ku * Jx / fu
    Yh = -lv * Jy / gv
    eu = np.where(np.arange(Mx) == 0, 1.0, 2.0)
    ev = np.where(np.arange(My) == 0, 1.0, 2.0)
    k2 = ku[:, None] ** 2 + lv[None, :] ** 2
    k2[0, 0] = 1.0
    G = eu[:, None] * ev[None, :] / (W * H * k2)
    G[0, 0] = 0.0
    a = G * fu[:, None] * gv[None, :] * mul_sum(Xs, Ys, prec)
    K = fu[:, None] * a * gv[None, :]
    T, Tp = mul_sum(Xs.T, K, prec), mul_sum(Xh.T, K, prec)      # X K, contraction over u
    N = np.sum(T * Ys, axis=1)
    gx = np.sum(Tp * Ys, axis=1)
    gy = np.sum(T * Yh, axis=1)
    S = np.where(G > 0, a / np.where(G > 0, G, 1.0), 0.0)
    return dict(a=a, N=N, gx=gx, gy=gy, E=0.5 * float(np.sum(a * S)))


CASES = [
    lambda: synth.out_of_die_blocks(300, 40, 33, seed=5, W=1.3, H=0.7),
    lambda: synth.uniform_blocks(500, 64, 48, seed=6, W=1.0, H=1.4, charge=True),
    lambda: synth.cell_mix(800, 72, 72, seed=7),
]


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_emulated_rounding_lies_inside_the_bound(prec, case):
    p = CASES[case]()
    ref = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    got = emulate(p, prec)
    r = bound_ratios(got, ref, p, prec, "rect")
    assert all(v <= 1.0 for v in r.values()), r
    # not vacuous: the operand rounding alone (the emulation has no generator or
    # accumulation error) uses a visible part of the bound
    assert r["a"] > 0.1 and max(r["N"], r["gx"], r["gy"]) > 0.03, r


def G0(p):
    ku = np.arange(p.Mx) * math.pi / p.W
    lv = np.arange(p.My) * math.pi / p.H
    eu = np.where(np.arange(p.Mx) == 0, 1.0, 2.0)
    ev = np.where(np.arange(p.My) == 0, 1.0, 2.0)
    k2 = ku[:, None] ** 2 + lv[None, :] ** 2
    k2[0, 0] = 1.0
    return eu[:, None] * ev[None, :] / (p.W * p.H * k2)


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_planted_mistakes_break_the_bound(prec):
    p = CASES[0]()
    ref = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    good = emulate(p, prec)
    sub = p.subset(np.arange(1, p.n))                       # one block dropped
    a_drop = O.coefficients(sub.W, sub.H, sub.x, sub.y, sub.w, sub.h, sub.c, p.Mx, p.My)
    a_flip = good["a"].copy()
    a_flip[3, :] *= -1.0                                     # one mode's sign
    N_shift = O.energy_grad(p.W, p.H, p.x, p.y, p.w, p.h, p.c, np.roll(ref["a"], 1, axis=0))[0]
    mistakes = {
        "dropped block": dict(good, a=a_drop),
        "flipped mode": dict(good, a=a_flip),
        "mode index shifted in N": dict(good, N=N_shift),
        "gradient sign": dict(good, gx=-good["gx"]),
        "energy without the 1/2": dict(good, E=2 * good["E"]),
        "energy without the u = 0 modes": dict(good, E=good["E"] - 0.5 * float(
            np.sum(ref["a"][0, 1:] ** 2 / G0(p)[0, 1:]))),
    }
    for what, out in mistakes.items():
        r = bound_ratios(out, ref, p, prec, "rect")
        assert max(r.values()) > 1.0, (what, r)
