"""Gradient-descent driver over block positions: a plain, fixed-step loop around the
density evaluation alone (the Sec. IV loop with wirelength, Nesterov steps and the
penalty schedule is `place.py`).

Each step evaluates E and its gradient through the C ABI, then moves the
movable blocks with pp_descent_step:  x <- clamp(x - lr * dE/dx + j, w/2, W - w/2)
(same for y), with a seed-fixed jitter j ~ N(0, (jitter * W)^2) per block and step
drawn on the device (Philox4x32-10 counted by (block, step), Box-Muller).

Chunked evaluation.  The coefficients are a sum over blocks (Eq. aup sums over
i), so with the blocks cut into chunks, a = sum_c a(chunk c), summed in FP64 on
the device by pp_coeffs_accumulate, and each chunk's gradients follow from
pp_grad with that total a; the total energy is 1/2 sum_uv a_uv S_uv of the total
a (pp_energy_from_coeffs).  This bounds the workspace by the chunk size for
placements too large for one call.
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
    a64 = torch.zeros((Mx, My), dtype=torch.float64, device=x.device)
    a = torch.empty((Mx, My), dtype=torch.float32, device=x.device)
    for k, (s, e) in enumerate(zip(cuts[:-1], cuts[1:])):
        last = k == len(cuts) - 2
        binding.coeffs_accumulate(x[s:e], y[s:e], w[s:e], h[s:e], sl(c, s, e), W, H, Mx, My, a64, prec,
                                  a_out=a if last else None)
    gx = torch.empty_like(x)
    gy = torch.empty_like(y)
    for s, e in zip(cuts[:-1], cuts[1:]):
        binding.grad(x[s:e], y[s:e], w[s:e], h[s:e], sl(c, s, e), W, H, Mx, My, prec, a=a,
                     out=(gx[s:e], gy[s:e], None, None))
    # E = 1/2 sum_uv a_uv S_uv from the summed coefficients (the whole placement's)
    return gx, gy, binding.energy_from_coeffs(a, W, H)


def block_energies_chunked(x, y, w, h, c, W, H, Mx, My, prec="tf32", chunk: Optional[int] = None):
    """Per-block energies N_i of the whole placement, chunked as evaluate_chunked."""
    n = x.numel()
    if not chunk or chunk >= n:
        return binding.energy(x, y, w, h, c, W, H, Mx, My, prec)[0]
    cuts = list(range(0, n, chunk)) + [n]
    sl = lambda t, a, b: None if t is None else t[a:b]
    a64 = torch.zeros((Mx, My), dtype=torch.float64, device=x.device)
    a = torch.empty((Mx, My), dtype=torch.float32, device=x.device)
    for k, (s, e) in enumerate(zip(cuts[:-1], cuts[1:])):
        binding.coeffs_accumulate(x[s:e], y[s:e], w[s:e], h[s:e], sl(c, s, e), W, H, Mx, My, a64, prec,
                                  a_out=a if k == len(cuts) - 2 else None)
    eb = torch.empty_like(x)
    for s, e in zip(cuts[:-1], cuts[1:]):
        eb[s:e] = binding.energy(x[s:e], y[s:e], w[s:e], h[s:e], sl(c, s, e), W, H, Mx, My, prec, a=a)[0]
    return eb


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
    res = DescentResult()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for k in range(steps):
        gx, gy, E = evaluate_chunked(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec, chunk)
        res.energy.append(E)
        if callback is not None:
            callback(k, x, y, gx, gy, E)
        binding.descent_step(x, y, w, h, gx, gy, p.W, p.H, lr, jitter * p.W, seed, k, movable=mov)
    t1.record()
    torch.cuda.synchronize()
    binding.sync_status(dev)
    res.energy = [float(e.item()) for e in res.energy]
    res.x, res.y = x, y
    res.ms_per_step = t0.elapsed_time(t1) / max(steps, 1)
    return res


def ulp_steps(x0: np.ndarray, x1: np.ndarray) -> np.ndarray:
    """(x1 - x0) in units of half the float32 ulp of x0, as exact int64 integers: a
    float32 x1 in the binade of x0 or an adjacent one is a multiple of that unit, so
    x1 = float32(x0 + k * spacing(x0) / 2) recovers it from x0 alone (checked here)."""
    x0 = np.asarray(x0, np.float32)
    x1 = np.asarray(x1, np.float32)
    unit = 0.5 * np.spacing(np.abs(x0)).astype(np.float64)
    k = (x1.astype(np.float64) - x0.astype(np.float64)) / unit
    ki = np.rint(k).astype(np.int64)
    if not np.array_equal(ki.astype(np.float64), k):
        raise ValueError("positions are not a whole number of units apart")
    return ki


def save_checkpoint(path: str, step: int, p, x, y, gx, gy, eb, E, sample, positions: bool):
    """A record of step `step` for a later FP64 check: the GPU's gradient and per-block
    energy on the sample blocks and E; with `positions`, every block's position as
    ulp steps from its starting position (lzma-compressed int32/int64)."""
    import lzma
    import os
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    idx = torch.from_numpy(sample).to(x.device)
    rec = {"step": step, "n": p.n, "Mx": p.Mx, "My": p.My, "E": float(E),
           "sample": sample.astype(np.int64), "gx": gx[idx].cpu().numpy(), "gy": gy[idx].cpu().numpy(),
           "N": eb[idx].cpu().numpy()}
    if positions:
        for name, start, now in (("dx", p.x, x), ("dy", p.y, y)):
            k = ulp_steps(start, now.cpu().numpy())
            dt = np.int32 if np.abs(k).max(initial=0) < 2 ** 31 else np.int64
            rec[name] = lzma.compress(k.astype(dt).tobytes(), preset=6)
            rec[name + "_dtype"] = np.dtype(dt).str
    np.savez(path, **{k: (np.frombuffer(v, np.uint8) if isinstance(v, bytes) else v) for k, v in rec.items()})


def _main(argv=None) -> int:
    """Run the descent loop on a synthetic workload and print one JSON line:
    time per step, block-mode^2 terms/s, the energy trace, and the same first
    evaluation in FP32 plain for comparison (time and relative gradient gap)."""
    import argparse
    import json
    ap = argparse.ArgumentParser(prog="python -m paper_2307_12041_gb300.descent")
    ap.add_argument("--workload", type=int, default=4, help="synth.WORKLOADS index")
    ap.add_argument("--n", type=int, default=None, help="first n blocks only")
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--lr", type=float, default=1e-4)
    ap.add_argument("--jitter", type=float, default=1e-6)
    ap.add_argument("--prec", default="tf32")
    ap.add_argument("--chunk", type=int, default=None)
    ap.add_argument("--fp32-steps", type=int, default=2, help="FP32-plain evaluations to time")
    ap.add_argument("--check-every", type=int, default=0,
                    help="also evaluate E in FP32 plain at the current positions every K steps")
    ap.add_argument("--save-dir", default=None,
                    help="save records for an FP64 check of the first and last steps (the GPU's "
                         "gradient and N on --sample blocks, E, and the last positions)")
    ap.add_argument("--sample", type=int, default=10000, help="sample blocks of the saved records")
    a = ap.parse_args(argv)
    p = synth.workload(a.workload, n=a.n)
    dev = torch.device("cuda")
    terms = float(p.n) * p.Mx * p.My
    descend(p, 2, a.lr, a.jitter, prec=a.prec, chunk=a.chunk)          # warm-up (workspaces, modules)
    checks = []
    if a.check_every:
        # a separate run (checks would perturb the timing): E in both precisions
        def cb(k, xk, yk, gxk, gyk, Ek):
            if k % a.check_every == 0:
                wk, hk, ck = binding.to_device(p, dev)[2:]
                Ep = evaluate_chunked(xk, yk, wk, hk, ck, p.W, p.H, p.Mx, p.My, "fp32", a.chunk)[2]
                checks.append((k, float(Ek.item()), float(Ep.item())))
        descend(p, a.steps, a.lr, a.jitter, prec=a.prec, chunk=a.chunk, callback=cb)
    saved = []
    if a.save_dir:
        # a separate run (saving would perturb the timing): records of the first and last steps
        import os
        sample = np.sort(np.random.default_rng(synth.BASE_SEED + 99).choice(p.n, min(a.sample, p.n),
                                                                           replace=False))
        last = a.steps - 1

        def cb_save(k, xk, yk, gxk, gyk, Ek):
            if k not in (0, last):
                return
            wk, hk, ck = binding.to_device(p, dev)[2:]
            ebk = block_energies_chunked(xk, yk, wk, hk, ck, p.W, p.H, p.Mx, p.My, a.prec, a.chunk)
            path = os.path.join(a.save_dir, f"step{k:03d}.npz")
            save_checkpoint(path, k, p, xk, yk, gxk, gyk, ebk, Ek.item(), sample, positions=k == last)
            saved.append(path)

        descend(p, a.steps, a.lr, a.jitter, prec=a.prec, chunk=a.chunk, callback=cb_save)
    res = descend(p, a.steps, a.lr, a.jitter, prec=a.prec, chunk=a.chunk)
    x, y, w, h, c = binding.to_device(p, dev)
    x, y = res.x, res.y                                 # compare at the final positions
    g_mixed = evaluate_chunked(x, y, w, h, c, p.W, p.H, p.Mx, p.My, a.prec, a.chunk)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(a.fp32_steps):
        g_plain = evaluate_chunked(x, y, w, h, c, p.W, p.H, p.Mx, p.My, "fp32", a.chunk)
    t1.record()
    torch.cuda.synchronize()
    binding.sync_status(dev)
    fp32_ms = t0.elapsed_time(t1) / max(a.fp32_steps, 1)
    scale = float(torch.maximum(g_plain[0].abs().max(), g_plain[1].abs().max()))
    gap = max(float((g_mixed[0] - g_plain[0]).abs().max()), float((g_mixed[1] - g_plain[1]).abs().max()))
    e = res.energy
    print(json.dumps({
        "workload": synth.WORKLOADS[a.workload]["name"], "n": p.n, "Mx": p.Mx, "My": p.My,
        "precision": a.prec, "steps": a.steps, "lr": a.lr, "jitter": a.jitter, "chunk": a.chunk,
        "ms_per_step": res.ms_per_step, "terms_per_s": terms / (res.ms_per_step / 1e3),
        "energy_first": e[0], "energy_last": e[-1],
        "energy_trace": [e[i] for i in range(0, len(e), max(1, len(e) // 10))] + [e[-1]],
        "fp32_plain_ms_per_eval": fp32_ms, "speedup_vs_fp32_plain": fp32_ms / res.ms_per_step,
        "grad_gap_vs_fp32_plain": gap / scale if scale > 0 else gap,
        "E_gap_vs_fp32_plain": abs(float(g_mixed[2]) - float(g_plain[2])) / abs(float(g_plain[2])),
        "E_checks": checks, "saved": saved,
    }), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(_main())
