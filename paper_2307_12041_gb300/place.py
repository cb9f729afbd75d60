"""The placement loop of Sec. IV around the density energy: minimise
    f(v) = W_LSE(v) + lambda N(v)
with one Nesterov step per iteration, a penalty update and an overflow stop.  The
paper takes the optimiser and its parameters from ePlace without restating them;
the readings used here (each a parameter of `place`):

* density N: the exact series of this library (`pp_grad`, rectangle reading, any
  precision), E = 1/2 sum_i N_i and its gradient; or, as in the paper's own placer,
  the binned fast scheme of Sec. III-D on M x M bins (`pp_binned_grad`, centre
  reading, FP32 or TF32 transforms);
* wirelength: log-sum-exp with smoothing gamma = 8 w_b 10^{(20/9)(tau - 0.1) - 1}
  (w_b the bin width, tau the current overflow: gamma shrinks as the placement
  spreads);
* initial penalty lambda_0 = sum_i |dW_i| / sum_i |dN_i| (L1 norms), then
  lambda <- mu lambda with mu = 1.1^{1 - dHPWL / dHPWL_ref} clamped to [0.75, 1.1]
  and dHPWL_ref = 3.5e-3 of the starting HPWL;
* gradient preconditioned by max(1, |nets of i| + lambda q_i) (q_i the block's
  area);
* step length |v_k - v_{k-1}| / |g_k - g_{k-1}| (first step: the largest gradient
  moves one bin width), Nesterov momentum from a_{k+1} = (1 + sqrt(4 a_k^2 + 1)) / 2;
* overflow on the M x M bins of the mode grid at target density 1, stop below
  tau_stop = 0.1;
* filler cells (optional, `fillers=True`): movable cells without nets, of the mean
  movable cell's size, as many as bring the total block area to target * W * H,
  started uniformly over the die; they take part in the density term only (not in
  the wirelength, nor in the overflow, which measures the given blocks).

Every per-iteration step runs in the library's kernels through the C ABI.  In the
host loop the host keeps the scalars (lambda, gamma, a_k) and reads one small vector
back per iteration (overflow, W_LSE, HPWL, E); in the device loop (the default after
the first iteration when no callback is given) the library makes the same scalar
updates on the device between iterations (pp_place_run, one CUDA graph with a
conditional WHILE node) and the host reads the records once, at the end.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import torch

from . import binding, synth


@dataclass
class PlaceResult:
    trace: List[dict] = field(default_factory=list)
    x: Optional[torch.Tensor] = None
    y: Optional[torch.Tensor] = None
    iterations: int = 0
    ms_per_iter: float = 0.0
    graph: bool = False                 # iterations after the first replayed a CUDA graph
    graph_error: Optional[str] = None   # why the capture failed, if it did
    device_loop: bool = False           # iterations after the first ran as one device-resident loop
    device_loop_error: Optional[str] = None   # why pp_place_run was refused, if it was
    stop: Optional[str] = None          # the device loop's stop code (converged, max_iters, ...)


def gamma_of(tau: float, bin_w: float) -> float:
    return 8.0 * bin_w * 10.0 ** ((20.0 / 9.0) * (tau - 0.1) - 1.0)


class Placer:
    """The loop's state on the device (major and reference solutions u, v, the
    previous v and gradient, the netlist, the bins) and its scalars (lambda,
    gamma, a_k); step() runs one iteration and returns its record.  After the
    first iteration (whose lambda_0 and step length need host reductions) each
    step is one library call, pp_place_iteration, and one 32-byte read-back;
    with graph=True that call is captured once in a CUDA graph and replayed with
    the iteration's lambda, gamma and momentum written to the device.
    fused=False issues the same kernels through the separate entry points."""

    def __init__(self, p: synth.Placement, net_ptr, net_pin, prec: str = "tf32", target: float = 1.0,
                 d_hpwl_frac: float = 3.5e-3, device="cuda", density: str = "exact", fillers: bool = False,
                 filler_seed: int = synth.BASE_SEED + 99, fused: bool = True, graph: bool = True):
        if density not in ("exact", "binned"):
            raise ValueError("density must be 'exact' or 'binned'")
        dev = torch.device(device)
        self.density = density
        self.n_real = p.n
        if fillers:
            p = with_fillers(p, target, filler_seed)
        self.p, self.prec, self.target, self.d_hpwl_frac = p, prec, target, d_hpwl_frac
        self.nl = binding.DeviceNetlist(p.n, net_ptr, net_pin, dev)
        x, y, self.w, self.h, self.c = binding.to_device(p, dev)
        self.M = p.Mx
        self.bin_w = p.W / self.M
        self.ux, self.uy = x.clone(), y.clone()
        self.vx, self.vy = x.clone(), y.clone()
        self.vpx, self.vpy = x.clone(), y.clone()
        self.gpx, self.gpy = torch.zeros_like(x), torch.zeros_like(y)
        self.q = self.w * self.h if self.c is None else self.c * self.w * self.h
        self.mov = None if p.movable is None else torch.from_numpy(p.movable.astype("uint8")).to(dev)
        nr = self.n_real                      # overflow and its area: the given blocks only
        q_real = self.q[:nr]
        self.area_mov = float(q_real.sum() if self.mov is None else q_real[self.mov[:nr].bool()].sum())
        self.bin_area = (p.W / self.M) * (p.H / self.M)
        self.norms = torch.zeros(2, dtype=torch.float64, device=dev)
        self.bins = torch.empty((self.M, self.M), dtype=torch.float32, device=dev)
        ovf = self.overflow_now()
        self.tau = float(ovf.item()) * self.bin_area / self.area_mov
        self.gamma = gamma_of(self.tau, self.bin_w)
        self.lam, self.a_k, self.hp_prev, self.d_ref, self.k = None, 1.0, None, None, 0
        self.fused, self.use_graph, self._it = fused, graph, None
        self.stop = None

    def overflow_now(self):
        nr = self.n_real
        ovf, _ = binding.overflow(self.ux[:nr], self.uy[:nr], self.w[:nr], self.h[:nr], self.p.W, self.p.H,
                                  self.M, self.target, bins=self.bins)
        return ovf

    def _fused(self) -> binding.PlaceIteration:
        if self._it is None:
            p = self.p
            dprec = self.prec if self.density == "exact" else ("fp32" if self.prec == "fp32" else "tf32")
            self._it = binding.PlaceIteration(self.nl, p.W, p.H, self.M, self.density, dprec, self.n_real,
                                              self.w, self.h, self.c, self.q, self.mov, self.ux, self.uy,
                                              self.vx, self.vy, self.vpx, self.vpy, self.gpx, self.gpy,
                                              self.target, graph=self.use_graph)
        return self._it

    def step(self) -> dict:
        p, M, k = self.p, self.M, self.k
        a_next = (1.0 + math.sqrt(4.0 * self.a_k * self.a_k + 1.0)) / 2.0
        coef = (self.a_k - 1.0) / a_next
        if k > 0 and self.fused:              # one library call for the whole iteration
            s = self._fused()(self.lam, self.gamma, coef).cpu()     # the one read-back of the iteration
        else:
            if self.density == "exact":
                gnx, gny, _, E = binding.grad(self.vx, self.vy, self.w, self.h, self.c, p.W, p.H, M, M,
                                              self.prec)
            else:                             # binned scheme: bins = modes per axis (K = m - 1)
                bprec = "fp32" if self.prec == "fp32" else "tf32"
                gnx, gny, _, E, _ = binding.binned_grad(self.vx, self.vy, self.w, self.h, self.c, p.W, p.H, M,
                                                        M, M, bprec, want_coeffs=False)
            gwx, gwy, wl = binding.wirelength(self.nl, self.vx, self.vy, self.gamma)
            if self.lam is None:              # lambda_0: ratio of the L1 gradient norms
                self.lam = float((gwx.abs().sum() + gwy.abs().sum()) / (gnx.abs().sum() + gny.abs().sum()))
            gx, gy = binding.place_combine(gwx, gwy, gnx, gny, self.nl.cell_ptr, self.q, self.mov, self.lam)
            if k > 0:
                binding.step_norms(self.vx, self.vy, self.vpx, self.vpy, gx, gy, self.gpx, self.gpy,
                                   self.norms)
                alpha0 = 0.0
            else:                             # first step: the largest gradient moves one bin
                gmax = float(torch.maximum(gx.abs().max(), gy.abs().max()))
                alpha0 = self.bin_w / gmax if gmax > 0 else 0.0
            binding.nesterov_step(p.W, p.H, self.ux, self.uy, self.vx, self.vy, self.vpx, self.vpy, gx, gy,
                                  self.gpx, self.gpy, self.w, self.h, self.mov,
                                  self.norms if k > 0 else None, alpha0, coef)
            ovf = self.overflow_now()
            s = torch.cat([ovf, wl, E.reshape(1)]).cpu()    # the one read-back of the iteration
        self.a_k = a_next
        self.tau = float(s[0]) * self.bin_area / self.area_mov
        rec = {"k": k, "tau": self.tau, "W_lse": float(s[1]), "hpwl": float(s[2]), "E": float(s[3]),
               "lambda": self.lam, "gamma": self.gamma}
        # penalty and smoothing updates for the next iteration
        if self.hp_prev is None:
            self.d_ref = self.d_hpwl_frac * rec["hpwl"]
        else:
            mu = 1.1 ** (1.0 - (rec["hpwl"] - self.hp_prev) / self.d_ref)
            self.lam *= min(1.1, max(0.75, mu))
        self.hp_prev = rec["hpwl"]
        self.gamma = gamma_of(self.tau, self.bin_w)
        self.k += 1
        return rec

    def run_device(self, iters: int, tau_stop: float) -> List[dict]:
        """Iterations k, k + 1, ... (k >= 1: the first step is the host's) on the device
        through pp_place_run, until tau < tau_stop or k = iters; the records in the
        format of step(), and the state (lambda, gamma, a_k, ...) taken back."""
        if self.k < 1 or self.lam is None or self.d_ref is None:
            raise RuntimeError("run_device continues a started loop: make the first step with step()")
        st = binding.PlaceState(lam=self.lam, gamma=self.gamma, a_k=self.a_k, hpwl_prev=self.hp_prev,
                                d_ref=self.d_ref, tau=self.tau, k=self.k, stop=0, run_count=0)
        sc = binding.PlaceSchedule(max_iters=int(iters), reserved=0, tau_stop=float(tau_stop),
                                   bin_area=self.bin_area, area_mov=self.area_mov, bin_w=self.bin_w)
        out, recs = self._fused().run(st, sc)
        self.lam, self.gamma, self.a_k, self.hp_prev = out.lam, out.gamma, out.a_k, out.hpwl_prev
        self.tau, self.k = out.tau, int(out.k)
        self.stop = binding.PLACE_STOP.get(int(out.stop), str(out.stop))
        return [{"k": int(r.k), "tau": r.tau, "W_lse": r.w_lse, "hpwl": r.hpwl, "E": r.e, "lambda": r.lam,
                 "gamma": r.gamma} for r in recs]


def with_fillers(p: synth.Placement, target: float, seed: int) -> synth.Placement:
    """p followed by filler cells (see the module notes): movable, no charge factor."""
    import numpy as np
    area = float(np.sum(p.w.astype(np.float64) * p.h))
    free = target * p.W * p.H - area
    mov = np.ones(p.n, bool) if p.movable is None else p.movable
    fw, fh = float(np.mean(p.w[mov])), float(np.mean(p.h[mov]))
    k = int(free // (fw * fh)) if free > 0 else 0
    if k == 0:
        return p
    g = np.random.default_rng(seed)
    fx = (0.5 * fw + g.random(k) * (p.W - fw)).astype(np.float32)
    fy = (0.5 * fh + g.random(k) * (p.H - fh)).astype(np.float32)
    cat = lambda a, b: np.concatenate([a, b]).astype(np.float32)
    c = None if p.c is None else cat(p.c, np.ones(k))
    return synth.Placement(p.W, p.H, cat(p.x, fx), cat(p.y, fy), cat(p.w, np.full(k, fw)),
                           cat(p.h, np.full(k, fh)), c, p.Mx, p.My,
                           movable=np.concatenate([mov, np.ones(k, bool)]), name=p.name + "+fillers",
                           meta=dict(p.meta, fillers=k))


def place(p: synth.Placement, net_ptr, net_pin, iters: int = 200, prec: str = "tf32",
          tau_stop: float = 0.1, target: float = 1.0, d_hpwl_frac: float = 3.5e-3,
          device="cuda", callback: Optional[Callable] = None, density: str = "exact",
          fillers: bool = False, fused: bool = True, graph: bool = True,
          device_loop: bool = True) -> PlaceResult:
    """Run up to `iters` iterations; callback(k, rec, x_eval, y_eval, ux, uy) after
    each, with the positions at which W_LSE and E of `rec` were evaluated.  With
    device_loop (and fused, and no callback) every iteration after the first runs in
    one pp_place_run call; if the library refuses it (res.device_loop_error says
    why) the host loop carries on from the same state."""
    pl = Placer(p, net_ptr, net_pin, prec, target, d_hpwl_frac, device, density, fillers, fused=fused,
                graph=graph)
    res = PlaceResult()
    dev = torch.device(device)
    use_dev = device_loop and fused and callback is None
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    while pl.k < iters:
        if use_dev and pl.k >= 1:
            try:
                recs = pl.run_device(iters, tau_stop)
            except binding.PPError as e:  # nothing ran: continue on the host
                res.device_loop_error, use_dev = str(e), False
                continue
            res.trace.extend(recs)
            res.device_loop, res.stop, res.iterations = True, pl.stop, pl.k
            break
        rec = pl.step()
        res.trace.append(rec)
        if callback is not None:          # vpx, vpy: the positions this iteration evaluated
            callback(rec["k"], rec, pl.vpx, pl.vpy, pl.ux, pl.uy)
        res.iterations = rec["k"] + 1
        if rec["tau"] < tau_stop:
            break
    torch.cuda.synchronize(dev)
    binding.sync_status(dev)
    res.ms_per_iter = (time.perf_counter() - t0) * 1e3 / max(res.iterations, 1)
    res.x, res.y = pl.ux[:pl.n_real], pl.uy[:pl.n_real]
    if pl._it is not None:
        res.graph, res.graph_error = pl._it.graph is not None, pl._it.graph_error
    return res


def _main(argv=None) -> int:
    """Run the loop on a synthetic netlist and print one JSON line: iterations,
    time per iteration, block-mode^2 terms/s of the density part, and the trace of
    overflow, HPWL and lambda."""
    import argparse
    import json
    ap = argparse.ArgumentParser(prog="python -m paper_2307_12041_gb300.place")
    ap.add_argument("--n", type=int, default=200_000)
    ap.add_argument("--modes", type=int, default=512)
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--prec", default="tf32")
    ap.add_argument("--seed", type=int, default=synth.BASE_SEED + 10)
    ap.add_argument("--density", choices=["exact", "binned"], default="exact")
    ap.add_argument("--fillers", action="store_true")
    ap.add_argument("--unfused", action="store_true", help="one entry point per step of an iteration")
    ap.add_argument("--no-graph", action="store_true", help="issue the fused call each iteration")
    ap.add_argument("--host-loop", action="store_true",
                    help="update the scalars on the host after each iteration instead of on the device")
    a = ap.parse_args(argv)
    p = synth.placement_cells(a.n, a.modes, a.seed)
    ptr, pins = synth.netlist(a.n, a.seed + 1)
    kw = dict(prec=a.prec, density=a.density, fillers=a.fillers, fused=not a.unfused, graph=not a.no_graph,
              device_loop=not a.host_loop)
    place(p, ptr, pins, iters=3, **kw)      # warm-up
    r = place(p, ptr, pins, iters=a.iters, **kw)
    t = r.trace
    pick = [t[i] for i in range(0, len(t), max(1, len(t) // 10))] + [t[-1]]
    print(json.dumps({
        "workload": p.name, "n": p.n, "nets": len(ptr) - 1, "pins": int(len(pins)), "modes": a.modes,
        "precision": a.prec, "density": a.density, "fillers": a.fillers, "fused": not a.unfused,
        "graph": r.graph, "graph_error": r.graph_error, "device_loop": r.device_loop,
        "device_loop_error": r.device_loop_error, "stop": r.stop,
        "iterations": r.iterations,
        "ms_per_iter": r.ms_per_iter,
        "density_terms_per_s": p.n * a.modes * a.modes / (r.ms_per_iter / 1e3),
        "tau_first": t[0]["tau"], "tau_last": t[-1]["tau"], "hpwl_first": t[0]["hpwl"],
        "hpwl_last": t[-1]["hpwl"],
        "trace": [{k: (round(v, 6) if isinstance(v, float) else v) for k, v in rec.items()} for rec in pick],
    }), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(_main())
