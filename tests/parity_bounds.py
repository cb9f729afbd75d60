"""Element-wise error bounds of the tensor-core precisions (test helper).

Used by the GPU parity tests next to the flat normalised bounds, and pinned on
the CPU by test_parity_bounds.py: an FP64 emulation of the kernels' operand
rounding lies inside the bound but uses a visible part of it, and planted
mistakes break it.

Model.  Each operand value of a contraction is rounded once, to nearest: TF32
keeps 11 significant bits (error up to 2^-11 |x|); BF16x3 represents x as
bf16 hi + lo (error up to 2^-18 |x|) and drops lo * lo (up to 2^-18 |x y|), taken
as 2^-17 per operand.  Such errors are independent and uniform, variance
(op |x|)^2 / 3 each (Higham, Accuracy and Stability of Numerical Algorithms,
Sec. 2.8 on statistical error analysis), so a contraction sum_k p_k q_k of rounded
operands has an error of standard deviation op sqrt(2/3 sum_k p_k^2 q_k^2), and
the bound is 6 such deviations (a sum of many small independent terms is close
to normal; for a single term, 6 deviations exceed the worst case 2 op |p q|).
Added to it:
 - the basis generators' sinusoid recurrences: an absolute error per value of at
   most gen * (the magnitude of the chain's values: |c_i| f_u (|sin(pi u t_i)| +
   min(1, pi (u + 32) t_i)) for the product of the centre and half-size chains,
   t_i = w_i / 2W), independent between blocks.  The largest such errors measured
   in FP32 emulation of the TF32 generators are 3.2e-5 (coefficient generator) and
   1e-5 (energy generator, epilogue); half of each is taken as the standard
   deviation (6 deviations: three times the largest error); the BF16x3 generators
   (Taylor anchors to 2e-9, then up to 32 rotation steps) take 1e-6;
 - the tensor cores' FP32 accumulation, which may truncate by one unit in the last
   place per MMA step, a bias (not random): steps * 2^-23 * (|result| + 3 RMS
   of the partial sums), with min(n, chain) / 8 steps per coefficient chain (TF32:
   8 blocks per step, chains of 8,192 blocks) or 3 min(n, 2048) / 16 (BF16x3), and
   Mx / 8 or 3 Mx / 16 per energy row;
 - the energy operand K = f a g: the coefficients' own error (variance of a)
   plus its rounding; the epilogue's row dots run in FP32 (4 units of |result|).
The magnitudes come from the FP64 oracle's rectangle integrals.
"""
import math

import numpy as np

from oracle import series as O

BOUND_PARAMS = {
    "tf32": dict(op=2.0 ** -11, gen_c=1.6e-5, gen_e=5e-6, chain=8192, kstep=8, mmas=1),
    "bf16x3": dict(op=2.0 ** -17, gen_c=1e-6, gen_e=1e-6, chain=2048, kstep=16, mmas=3),
}
ULP32 = 2.0 ** -23
SIGMAS = 6.0


def _np(t):
    return t.double().cpu().numpy() if hasattr(t, "cpu") else np.asarray(t, np.float64)


def error_bounds(ref, p, prec, sample="rect"):
    """Per-element error bounds {a, N, gx, gy: arrays, E: float} of the GPU result
    in precision `prec` against the oracle result `ref` of placement `p`."""
    P = BOUND_PARAMS[prec]
    r3 = P["op"] ** 2 / 3.0
    W, H, n, Mx, My = float(p.W), float(p.H), p.n, p.Mx, p.My
    x, y, w, h = (np.asarray(v, np.float64) for v in (p.x, p.y, p.w, p.h))
    cc = np.ones(n) if p.c is None else np.asarray(p.c, np.float64)
    ku = np.arange(Mx) * math.pi / W
    lv = np.arange(My) * math.pi / H
    fu = 2.0 * W / (math.pi * np.maximum(np.arange(Mx), 1))
    gv = 2.0 * H / (math.pi * np.maximum(np.arange(My), 1))
    Ix, Jx = O.rect_integrals(x, w, W, Mx)
    Iy, Jy = O.rect_integrals(y, h, H, My)
    eu = np.where(np.arange(Mx) == 0, 1.0, 2.0)
    ev = np.where(np.arange(My) == 0, 1.0, 2.0)
    k2 = ku[:, None] ** 2 + lv[None, :] ** 2
    k2[0, 0] = 1.0
    G = eu[:, None] * ev[None, :] / (W * H * k2)
    G[0, 0] = 0.0
    a = np.asarray(ref["a"], np.float64)
    S = np.where(G > 0, a / np.where(G > 0, G, 1.0), 0.0)

    # coefficients: a = G o (X^T Y), X = c Ix, Y = Iy
    X, Y = cc[:, None] * Ix, Iy
    X2, Y2 = X * X, Y * Y
    # magnitude of the generators' chains: the centre chain's values are at most 1,
    # the half-size chain's |sin(pi u t)|, which it reaches through at most 32 modes
    # from an anchor (values up to min(1, pi (u + 32) t))
    def chain_amp(size, L, M):
        t = np.abs(np.asarray(size, np.float64))[:, None] / (2 * L)
        u = np.arange(M)[None, :]
        return np.abs(np.sin(math.pi * u * t)) + np.minimum(1.0, math.pi * (u + 32) * t)
    ampX = np.abs(cc)[:, None] * fu[None, :] * chain_amp(w, W, Mx)
    ampY = gv[None, :] * chain_amp(h, H, My)
    ampX2, ampY2 = ampX * ampX, ampY * ampY
    XY2 = X2.T @ Y2
    # per value: variance of its error (rounding + generator); the product of two
    # errors (second order) matters only where both bases vanish for every block
    # (u t_i and v t'_i integers: grid-aligned sizes)
    EX2 = r3 * X2 + P["gen_c"] ** 2 * ampX2
    EY2 = r3 * Y2 + P["gen_c"] ** 2 * ampY2
    var_a = G * G * (EX2.T @ (Y2 + EY2) + X2.T @ EY2)
    steps_a = P["mmas"] * math.ceil(min(n, P["chain"]) / P["kstep"]) + 2
    da = SIGMAS * np.sqrt(var_a) + steps_a * ULP32 * (np.abs(a) + 3 * G * np.sqrt(XY2)) \
        + 4 * ULP32 * np.abs(a)

    # energy and gradient: rows of (basis a basis^T) in the chosen reading
    if sample == "rect":
        BX, BY = X, Y
        BXp, BYp = cc[:, None] * ku[None, :] * Jx, lv[None, :] * Jy
        aX, aY = ampX, ampY
    else:
        q = cc * w * h
        BX, BY = q[:, None] * np.cos(np.outer(x, ku)), np.cos(np.outer(y, lv))
        BXp = q[:, None] * ku[None, :] * np.sin(np.outer(x, ku))
        BYp = lv[None, :] * np.sin(np.outer(y, lv))
        aX, aY = np.broadcast_to(np.abs(q)[:, None], BX.shape), np.ones(BY.shape)
    aXp, aYp = aX * ku[None, :], aY * lv[None, :]
    varK = var_a + r3 * a * a
    steps_e = P["mmas"] * math.ceil(Mx / P["kstep"]) + 2
    ge2 = P["gen_e"] ** 2

    def rows(Xb, ampx, Yb, ampy):
        R = Yb @ a.T                       # R_iu = sum_v a_uv Y_iv
        T = Xb @ a                         # T_iv = sum_u X_iu a_uv
        X2b, Y2b = Xb * Xb, Yb * Yb
        var = (r3 * np.sum(X2b * R * R, axis=1) + ge2 * np.sum(ampx * ampx * R * R, axis=1)
               + np.einsum("iu,uv,iv->i", X2b, varK, Y2b) + ge2 * np.sum(T * T * ampy * ampy, axis=1))
        rmsT = np.sqrt(X2b @ (a * a))
        bias = steps_e * ULP32 * np.sum((np.abs(T) + 3 * rmsT) * np.abs(Yb), axis=1)
        return SIGMAS * np.sqrt(var), var, bias

    sN, vN, bN = rows(BX, aX, BY, aY)
    sX, _, bX = rows(BXp, aXp, BY, aY)
    sY, _, bY = rows(BX, aX, BYp, aYp)
    out = {"a": da}
    for k, s_, b_ in (("N", sN, bN), ("gx", sX, bX), ("gy", sY, bY)):
        out[k] = s_ + b_ + 4 * ULP32 * np.abs(np.asarray(ref[k], np.float64))
    var_E = float(np.sum(S * S * var_a)) + 0.25 * float(np.sum(vN))
    out["E"] = (SIGMAS * math.sqrt(var_E) + float(np.sum(np.abs(S) * (da - SIGMAS * np.sqrt(var_a))))
                + 0.5 * float(np.sum(bN)) + 1e-9 * abs(ref["E"]))
    return out


def bound_ratios(out, ref, p, prec, sample="rect"):
    """max over elements of |gpu - oracle| / bound for a, N, gx, gy and E."""
    B = error_bounds(ref, p, prec, sample)
    r = {}
    for k in ("a", "N", "gx", "gy"):
        got = _np(out[k]).reshape(np.shape(ref[k]))
        r[k] = float(np.max(np.abs(got - ref[k]) / (B[k] + 1e-300)))
    dE = abs(float(out["E"]) - ref["E"])
    r["E"] = dE / B["E"] if B["E"] > 0 else (0.0 if dE == 0 else math.inf)
    return r
