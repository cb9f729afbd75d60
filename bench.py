#!/usr/bin/env python3
"""Throughput of one energy + gradient evaluation of the analytical Poisson series.

Metric: block * mode^2 terms per second, N * Mx * My / t, where t is the device
time of one full evaluation through the C ABI (pp_grad with a = NULL: the
coefficient contraction, the two energy contractions, the row dots, per-block
energies and the FP64 total), mixed precision next to FP32 plain, with the
error against the FP64 oracle.

Workload: 200,000 blocks on a 1 x 1 die (99% standard cells h = 0.001,
w lognormal mean 0.002; 1% macros 0.01-0.05; centres from 20 Gaussian
clusters), 512 x 512 modes.  Seeded synthetic data (the paper's ISPD placements
are not available).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec tf32|bf16x3|fp32]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)

Under torchrun (N > 1) the ranks share one placement of N x 200,000 blocks
(each rank's 200,000 blocks; per-GPU work fixed, weak scaling): per step every
rank adds its blocks' coefficients into an FP64 array, one all-reduce sums it
over the ranks, and every rank evaluates its own blocks against the whole
placement's coefficients; the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "block·mode² terms/s for energy+gradient, mixed vs FP32, err vs FP64"
WORKLOAD_INDEX = 1
FLUSH_BYTES = 256 << 20          # > 129 MB L2
FP32_LANES_PER_SM = 128
SM_COUNT_GB300 = 152


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# tensor-core kernels on this workload, from one ncu capture of the bench command
# (profiles/tc_traffic_cellmix-200k-512x512.md), valid only while the kernel sources
# hash to the digest they were captured with, and only for that workload (its
# block·mode² terms N Mx My).
NCU_TRAFFIC = {
    "terms": 200_000 * 512 * 512,
    "digest": "224fa4164969ab3b",
    ("tf32", "coeff"): 25.636096e6 + 0.367616e6,
    ("tf32", "energy"): 26.693632e6 + 0.0,
}


# the sources of the tensor-core kernels (their code, layouts and launch plans)
TC_SOURCES = ("pp_tc.cu", "pp_tc.cuh", "pp_gen.cuh", "pp_device.cuh", "pp_internal.h")


def kernel_source_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in TC_SOURCES:
        h.update(name.encode())
        with open(os.path.join(ROOT, "paper_2307_12041_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(prec: str, kernel: str, terms: float):
    if kernel_source_digest() != NCU_TRAFFIC["digest"] or terms != NCU_TRAFFIC["terms"]:
        return None
    return NCU_TRAFFIC.get((prec, kernel))


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            return None
        rows = []
        for line in out.strip().splitlines():
            f = [s.strip() for s in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(f[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                rows.append(dict(ts=ts, sm=float(f[2]), max=float(f[3]), reasons=f[5],
                                 hw=f[6], hwt=f[7], swt=f[8], pcap=f[9]))
            except Exception:
                continue
        if not rows:
            return None
        inside = [r for r in rows if self.t0 - 1 <= r["ts"] <= self.t1 + 1] or rows
        reasons = set()
        for r in inside:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in inside),
                "sm_max_mhz": max(r["max"] for r in inside),
                "reasons": sorted(reasons), "samples": len(inside)}


# ---------------------------------------------------------------------------
# distributed plumbing (replicas)
# ---------------------------------------------------------------------------
def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend)
    return dist


def reduce_max(value: float, world: int, device=None) -> float:
    """Maximum of `value` over ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_throughput(units_per_rank: float, steps: int, rank_ms: float, world: int,
                         device=None):
    """(units/s over all ranks, slowest rank's ms): every rank processes
    `units_per_rank` per step; the job takes as long as its slowest rank."""
    total_ms = reduce_max(rank_ms, world, device)
    return world * units_per_rank * steps / (total_ms / 1e3), total_ms


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# the step
# ---------------------------------------------------------------------------
def make_inputs(device, n=None, workload=WORKLOAD_INDEX, mode="grad", world=1, rank=0):
    import torch
    from paper_2307_12041_gb300 import sharded, synth
    p = synth.workload(workload, n=n)
    if mode == "place":         # the loop's inputs: cells at 70% utilisation, started in a cluster
        p = synth.placement_cells(p.n, p.Mx, synth.BASE_SEED + 10 + workload)
    if mode == "sharded":       # one placement of world x n blocks, this rank's contiguous share
        whole = synth.workload(workload, n=world * p.n)
        p = sharded.shard(whole, world, rank)
        p.name = f"{synth.WORKLOADS[workload]['name']} x{world} blocks, sharded"
    t = lambda a: torch.from_numpy(a).to(device)
    return p, (t(p.x), t(p.y), t(p.w), t(p.h), None)


def time_steps(binding, p, dev_in, prec, steps, warmup, flush, outs, kernel_timing=False,
               mode="grad", bins=None):
    """Per-step CUDA-event times (ms) of `steps` evaluations after `warmup`; the L2
    is flushed (FLUSH_BYTES written) before every step, outside the events.  With
    kernel_timing, the library brackets each of its launches in the timed steps
    with events on the launch stream; returns (step times, per-kernel times).
    mode "grad": one pp_grad call (a computed inside); "autograd": the autograd
    function's forward (pp_energy) and backward (pp_grad, a recomputed), fixed
    blocks masked; "block-adjoint": per-block energies forward and the backward for
    a random upstream gradient (two coefficient and two energy contractions);
    "binned": the binned fast scheme (Sec. III-D) on `bins` x `bins` bins; "place": one
    iteration of the Sec. IV placement loop per step."""
    import torch
    x, y, w, h, c = dev_in
    stream = torch.cuda.current_stream()
    if mode in ("autograd", "block-adjoint"):
        mov = None if p.movable is None else torch.from_numpy(p.movable).to(x.device)
        xg = x.detach().clone().requires_grad_(True)
        yg = y.detach().clone().requires_grad_(True)
        gw = torch.randn(p.n, generator=torch.Generator().manual_seed(5), dtype=torch.float32).to(x.device)

        def run():
            xg.grad = None
            yg.grad = None
            if mode == "autograd":
                E = binding.PoissonEnergy.apply(xg, yg, w, h, c, p.W, p.H, p.Mx, p.My, prec, "rect", mov)
                E.backward()
            else:       # per-block energies, backward for an arbitrary upstream gradient
                N = binding.PoissonBlockEnergies.apply(xg, yg, w, h, c, p.W, p.H, p.Mx, p.My, prec, mov)
                N.backward(gw)
    elif mode == "place":        # one iteration of the Sec. IV loop per step (the loop's state carries over)
        from paper_2307_12041_gb300 import place as placemod, synth
        ptr, pins = synth.netlist(p.n, synth.BASE_SEED + 11)
        # the fused library call per iteration, not its CUDA-graph replay: the library
        # counts launches as they are issued, and a replay issues none from the host
        # (for this exact-density loop the two take the same time per iteration)
        placer = placemod.Placer(p, ptr, pins, prec, graph=False)
        run = placer.step
    elif mode == "sharded":      # this rank's blocks of one placement: one FP64 all-reduce per step
        from paper_2307_12041_gb300 import sharded
        run = lambda: sharded.evaluate(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec)
    elif mode == "binned":
        m = max(p.Mx, p.My) if bins is None else bins
        bprec = "tf32" if prec == "bf16x3" else prec
        run = lambda: binding.binned_grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, m, bprec, want_coeffs=False)
    else:
        run = lambda: binding.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec, out=outs)
    for _ in range(warmup):
        flush.zero_()
        run()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    binding.timing_collect()              # launch counts (and times) from here on
    if kernel_timing:
        binding.timing_enable(True)
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        run()
        b.record(stream)
    torch.cuda.synchronize()
    binding.timing_enable(False)
    ktimes = binding.timing_collect()     # {kernel: (launches, ms)}; ms 0 without kernel_timing
    binding.sync_status()
    return [a.elapsed_time(b) for a, b in evs], ktimes


def time_e2e(binding, p, prec, steps, device, flush, mode="grad", bins=None):
    """Same evaluation through host buffers, inside each step's CUDA events: x, y,
    w, h come from pinned host memory and gx, gy, N, E go back to pinned host
    memory.  mode "grad": one pp_grad_host call per step (its kernels read the
    inputs and write the outputs in place through the host link; E is copied out);
    the other modes copy the inputs in and the outputs out around their device
    call.  The L2 is flushed before every step, outside the events, as in the
    device-side timing."""
    import torch
    n = p.n
    hin = [torch.from_numpy(a).pin_memory() for a in (p.x, p.y, p.w, p.h)]
    din = [torch.empty(n, dtype=torch.float32, device=device) for _ in range(4)]
    dout = (torch.empty(n, dtype=torch.float32, device=device),
            torch.empty(n, dtype=torch.float32, device=device),
            torch.empty(n, dtype=torch.float32, device=device),
            torch.empty(1, dtype=torch.float64, device=device))
    hout = (torch.empty(n, dtype=torch.float32).pin_memory(),
            torch.empty(n, dtype=torch.float32).pin_memory(),
            torch.empty(n, dtype=torch.float32).pin_memory(),
            torch.empty(1, dtype=torch.float64).pin_memory())
    stream = torch.cuda.current_stream(device)

    def step():
        if mode == "grad":
            # the C-ABI call on host buffers: pinned inputs read and outputs written in
            # place by the kernels over the host link, E copied out
            binding.grad_host(hin[0], hin[1], hin[2], hin[3], None, p.W, p.H, p.Mx, p.My, prec,
                              out=hout, device=device)
            return
        for d, hsrc in zip(din, hin):
            d.copy_(hsrc, non_blocking=True)
        if mode == "sharded":
            from paper_2307_12041_gb300 import sharded
            gx, gy, eb, et, _ = sharded.evaluate(din[0], din[1], din[2], din[3], None, p.W, p.H, p.Mx, p.My,
                                                 prec)
            res = (gx, gy, eb, et)
        elif mode == "binned":
            gx, gy, eb, et, _ = binding.binned_grad(din[0], din[1], din[2], din[3], None, p.W, p.H, p.Mx, p.My,
                                                    bins, "tf32" if prec == "bf16x3" else prec,
                                                    want_coeffs=False)
            res = (gx, gy, eb, et)
        else:
            binding.grad(din[0], din[1], din[2], din[3], None, p.W, p.H, p.Mx, p.My, prec, out=dout)
            res = dout
        for hdst, d in zip(hout, res):
            hdst.copy_(d, non_blocking=True)

    for _ in range(3):
        step()
    torch.cuda.synchronize(device)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize(device)
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    h2d = 4 * 4 * n
    d2h = 3 * 4 * n + 8
    return ms, h2d, d2h


def errors_vs(ref, got):
    """Per output: max |err| / max |ref| and RMS err / RMS ref; the gradient also as
    one vector (both components normalised by the larger component scale)."""
    out = {}
    for k in ("a", "N", "gx", "gy"):
        r = np.asarray(ref[k], dtype=np.float64)
        g = np.asarray(got[k], dtype=np.float64).reshape(r.shape)
        d = g - r
        out[k] = {"max": float(np.max(np.abs(d)) / np.max(np.abs(r))),
                  "rms": float(np.sqrt(np.mean(d * d)) / np.sqrt(np.mean(r * r)))}
    r = np.stack([np.asarray(ref["gx"], np.float64), np.asarray(ref["gy"], np.float64)])
    g = np.stack([np.asarray(got["gx"], np.float64).reshape(-1), np.asarray(got["gy"], np.float64).reshape(-1)])
    d = g - r
    out["grad"] = {"max": float(np.max(np.abs(d)) / np.max(np.abs(r))),
                   "rms": float(np.sqrt(np.mean(d * d)) / np.sqrt(np.mean(r * r)))}
    out["E"] = abs(got["E"] - ref["E"]) / abs(ref["E"])
    return out


def cpu_baseline(binding, precs, device, n_sample, workload=WORKLOAD_INDEX):
    """The FP64 oracle as it stands on the host cores, on the first `n_sample`
    blocks of the workload (all modes), plus the GPU's error on that sample."""
    from oracle import series as O
    from paper_2307_12041_gb300 import synth
    full_n = synth.WORKLOADS[workload]["n"]
    n_sample = min(n_sample, full_n)
    p = synth.workload(workload).subset(np.arange(n_sample))
    cores = int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))
    t0 = time.perf_counter()
    ref = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    dt = time.perf_counter() - t0
    errs = {}
    for prec in precs:
        out = binding.evaluate(p, prec=prec, device=device)
        got = {k: out[k].double().cpu().numpy() for k in ("a", "N", "gx", "gy")}
        got["E"] = out["E"]
        errs[prec] = errors_vs(ref, got)
    base = {"value": n_sample * p.Mx * p.My / dt, "unit": "terms/s", "cores": cores,
            "kind": "oracle", "seconds": dt,
            "sample": f"first {n_sample} of {full_n} blocks, "
                      f"all {p.Mx}x{p.My} modes: coefficients, per-block energy, gradient (FP64 numpy)"}
    return base, errs


def oracle_single_core(workload, n_sample):
    """The oracle, as it stands, on ONE host core (the paper's setting: one CPU
    thread), on the first `n_sample` blocks of the workload: a child process pinned
    to one core with every BLAS / OpenMP pool limited to one thread."""
    code = ("import os, sys, time, json, numpy as np\n"
            "sys.path.insert(0, %r)\n"
            "from oracle import series as O\n"
            "from paper_2307_12041_gb300 import synth\n"
            "p = synth.workload(%d).subset(np.arange(%d))\n"
            "t0 = time.perf_counter()\n"
            "O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)\n"
            "dt = time.perf_counter() - t0\n"
            "print(json.dumps({'seconds': dt, 'n': p.n, 'Mx': p.Mx, 'My': p.My}))\n"
            % (ROOT, workload, n_sample))
    env = dict(os.environ, ORACLE_THREADS="1", OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1", BLIS_NUM_THREADS="1")

    def pin():
        try:
            os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})
        except (AttributeError, OSError):
            pass

    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, preexec_fn=pin,
                           capture_output=True, text=True, timeout=600, check=True)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:          # reported, not fatal: the GPU numbers stand on their own
        return {"error": f"{type(e).__name__}: {e}"}
    from paper_2307_12041_gb300 import synth
    full_n = synth.WORKLOADS[workload]["n"]
    return {"value": d["n"] * d["Mx"] * d["My"] / d["seconds"], "unit": "terms/s", "cores": 1,
            "seconds": d["seconds"],
            "sample": f"first {d['n']} of {full_n} blocks, all {d['Mx']}x{d['My']} modes, one core "
                      f"(process pinned to one CPU, BLAS and oracle threads 1)"}


def roofline(prec, ktimes, terms, peaks, peak_src):
    """Roofline of the slower of the coefficient and energy kernels: algorithmic
    flops per launch (2 or 4 N Mx My) over its average CUDA-event duration, against
    the measured peak of the precision's arithmetic."""
    dom = max(("coeff", "energy"), key=lambda k: ktimes[k][1])
    dom_ms = ktimes[dom][1] / max(ktimes[dom][0], 1)
    if dom_ms <= 0:
        return None
    flops = (2.0 if dom == "coeff" else 4.0) * terms
    if prec == "fp32":
        bound = "alu"
        peak = SM_COUNT_GB300 * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        note = f"FP32 FMA: {SM_COUNT_GB300} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x max SM clock"
    elif prec == "tf32":
        bound = "tensor"
        peak = peaks["bf16_tflops"] * 0.5
        note = f"{peak_src} bf16 burst peak x 0.5 (nominal TF32/BF16 ratio)"
    else:
        bound = "tensor"
        peak = peaks["bf16_tflops"] / 3.0
        note = f"{peak_src} bf16 burst peak / 3 (three bf16 products per term)"
    achieved = flops / (dom_ms * 1e-3) / 1e12
    return {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": ncu_traffic(prec, dom, terms), "peak_source": note,
            "flops_per_launch": flops, "kernel_ms": dom_ms}


def run_ours(args):
    import torch
    from paper_2307_12041_gb300 import binding, synth

    world, rank, local = dist_info()
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    if args.mode is None:       # one placement shared out over the ranks when there are several
        args.mode = "grad" if world == 1 else "sharded"
    device = torch.device("cuda", local)
    binding.lib()
    avail = binding.available_precisions()
    prec = args.prec or ("tf32" if "tf32" in avail else "fp32")
    if prec not in avail:
        raise SystemExit(f"precision {prec} not available: {avail}")
    # the precision the 1e-4 accuracy target binds, timed in the same run on the
    # same workload (its own line object; the headline `value` stays `prec`)
    extra = [q for q in ("bf16x3",) if q != prec and q in avail and args.mode in ("grad", "sharded")]

    p, dev_in = make_inputs(device, workload=args.workload, mode=args.mode, world=world, rank=rank)
    n = p.n
    outs = (torch.empty(n, dtype=torch.float32, device=device),
            torch.empty(n, dtype=torch.float32, device=device),
            torch.empty(n, dtype=torch.float32, device=device),
            torch.empty(1, dtype=torch.float64, device=device))
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=device)
    terms = float(n) * p.Mx * p.My

    def measure(q):
        # the headline steps run without per-launch events (they cost device time between
        # launches and stop each kernel from overlapping the previous one's tail); a second
        # pass of the same W + K steps brackets every launch with events for the kernel times
        ms, cnt = time_steps(binding, p, dev_in, q, args.steps, args.warmup, flush, outs,
                             mode=args.mode, bins=args.bins)
        kt = None
        if args.mode != "binned":
            _, kt = time_steps(binding, p, dev_in, q, args.steps, args.warmup, flush, outs,
                               kernel_timing=True, mode=args.mode, bins=args.bins)
        return ms, cnt, kt

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    clocks.mark("t0")
    step_ms, counts, ktimes = measure(prec)
    extra_runs = {q: measure(q) for q in extra}
    clocks.mark("t1")
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()

    value, total_ms = whole_job_throughput(terms, args.steps, sum(step_ms), world, device)
    ms_per_step = total_ms / args.steps

    peaks, peak_src = load_peaks()
    if ktimes is None:      # binned mode: the library's counters do not count these kernels
        ktimes = {"coeff": (0, 0.0), "energy": (0, 0.0)}
        m = args.bins or max(p.Mx, p.My)
        # density and interpolation (n > 0); the row prefix sums of the difference array
        # (FP32 atomics: n > 0 and m not 512 or 1024, else folded into the first row
        # transform; exact fixed-point density (fp32): always, with its conversion); FFT
        # tables (m a power of two); 7 row transforms (those followed by a step along the
        # other axis write transposed; for m = 512, 1024 the independent ones share a
        # launch: 4 launches); scaling
        warp = m in (512, 1024)
        prefix = 1 if prec == "fp32" else (1 if (p.n > 0 and not warp) else 0)
        per_step = (2 if p.n > 0 else 0) + prefix + (1 if m & (m - 1) == 0 else 0) + (4 if warp else 7) + 1
        launches = per_step * args.steps
    else:
        launches = int(sum(v[0] for v in counts.values()))     # our kernels in the timed steps
    extra_lines = {}
    for q, (q_ms, q_cnt, q_kt) in extra_runs.items():
        q_value, q_total = whole_job_throughput(terms, args.steps, sum(q_ms), world, device)
        extra_lines[q] = {"value": q_value, "unit": "terms/s", "ms_per_step": q_total / args.steps,
                          "gpu_launches": int(sum(v[0] for v in q_cnt.values())),
                          "roofline": roofline(q, q_kt, terms, peaks, peak_src),
                          "kernels_ms_per_step": {k: v[1] / args.steps for k, v in q_kt.items()}}

    line = {
        "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec,
        "data": "synthetic",
        "config": {"workload": p.name if args.mode in ("place", "sharded") else synth.WORKLOADS[args.workload]["name"],
                   "mode": args.mode,
                   "bins": (args.bins or max(p.Mx, p.My)) if args.mode == "binned" else None, "n": n, "Mx": p.Mx,
                   "My": p.My, "sample": "rect", "precision": prec, "W": p.W, "H": p.H,
                   "l2": "flushed: 256 MiB written before every timed step",
                   "kernel_times": "per-launch CUDA events in a second pass of the same steps",
                   "parallelism": (f"blocks sharded over {world} ranks (one FP64 all-reduce of the "
                                   f"{p.Mx} x {p.My} coefficient sums per step)") if args.mode == "sharded"
                                  else f"replicas x{world}"},
        "roofline": roofline(prec, ktimes, terms, peaks, peak_src),
        "kernels_ms_per_step": {k: v[1] / args.steps for k, v in ktimes.items()},
        "gpu_launches": launches + sum(v["gpu_launches"] for v in extra_lines.values()),
        "clocks": clk,
    }
    line.update(extra_lines)
    # end to end through host buffers: every rank (the sharded evaluation holds a collective)
    barrier(world)
    e_mode = args.mode if args.mode in ("grad", "sharded", "binned") else "grad"
    e_ms, h2d, d2h = time_e2e(binding, p, prec, args.steps, device, flush, mode=e_mode,
                              bins=args.bins or max(p.Mx, p.My))
    e_ms = reduce_max(e_ms, world, device)
    line["e2e"] = {"value": world * terms / (e_ms / 1e3), "unit": "terms/s",
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "ms_per_step": e_ms, "mode": e_mode,
                   "call": ("pp_grad_host: pinned host inputs read and outputs written in place by the kernels"
                            if e_mode == "grad" else "cudaMemcpyAsync in, device call, cudaMemcpyAsync out")}
    if rank == 0:
        # FP32 plain on the same workload (the "vs FP32" half of the metric); in sharded
        # mode on rank 0's blocks alone, with no collective (the other ranks wait)
        if prec != "fp32":
            torch.cuda.synchronize()
            f_mode = "grad" if args.mode == "sharded" else args.mode
            f_ms, _ = time_steps(binding, p, dev_in, "fp32", args.steps, args.warmup, flush, outs,
                                 mode=f_mode, bins=args.bins)
            fv = terms * args.steps / (sum(f_ms) / 1e3)
            line["fp32_plain"] = {"value": fv, "ms_per_step": sum(f_ms) / args.steps,
                                  "speedup_of_mixed": value / world / fv}
            for q, ql in extra_lines.items():
                ql["speedup_over_fp32_plain"] = ql["value"] / world / fv
        if world == 1 and not args.no_cpu_baseline:
            precs = [prec] + extra + (["fp32"] if prec != "fp32" else [])
            base, errs = cpu_baseline(binding, precs, device, args.cpu_sample, args.workload)
            base["single_core"] = oracle_single_core(args.workload, args.cpu_sample_1core)
            line["cpu_baseline"] = base
            line["errors_vs_fp64_oracle"] = {"sample": base["sample"], **errs}
            for q, ql in extra_lines.items():
                ql["errors_vs_fp64_oracle"] = errs[q]
        print(json.dumps(line), flush=True)
    barrier(world)


def run_reference(args):
    """The FP64 oracle, unmodified, on the host cores: each step evaluates the same
    workload (or, with --ref-sample, its first blocks), all modes."""
    world, rank, _ = dist_info()
    if rank != 0:
        return
    from oracle import series as O
    from paper_2307_12041_gb300 import synth
    full_n = synth.WORKLOADS[args.workload]["n"]
    n_s = min(args.ref_sample or full_n, full_n)
    p = synth.workload(args.workload).subset(np.arange(n_s))
    for _ in range(args.warmup):
        O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    dt = time.perf_counter() - t0
    terms = float(n_s) * p.Mx * p.My
    value = terms * args.steps / dt
    cores = int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))
    sample = (f"the whole workload ({full_n} blocks, {p.Mx}x{p.My} modes) per step" if n_s == full_n else
              f"first {n_s} of {full_n} blocks, all {p.Mx}x{p.My} modes, per step")
    line = {"metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": synth.WORKLOADS[args.workload]["name"], "n": p.n,
                       "Mx": p.Mx, "My": p.My, "sample": "rect", "precision": "f64"},
            "cpu_baseline": {"value": value, "unit": "terms/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "terms/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--prec", choices=["fp32", "tf32", "bf16x3"], default=None)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-sample", type=int, default=200000)
    ap.add_argument("--ref-sample", type=int, default=None,
                    help="blocks per reference step (default: the whole workload, ~4.4 s per step on "
                         "16 host cores at 200k x 512^2)")
    ap.add_argument("--cpu-sample-1core", type=int, default=20000,
                    help="blocks of the one-core oracle timing (the paper's single-thread setting)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", type=int, default=WORKLOAD_INDEX,
                    help="synth.WORKLOADS index (default: the metric's 200k x 512^2 workload)")
    ap.add_argument("--bins", type=int, default=None, help="bins per side for --mode binned")
    ap.add_argument("--mode", choices=["grad", "sharded", "autograd", "block-adjoint", "binned", "place"],
                    default=None,
                    help="default: grad on one GPU, sharded on several; "
                         "grad: one pp_grad per step; sharded: one placement of N x the workload's blocks "
                         "shared out over the N ranks (pp_coeffs_accumulate, an FP64 all-reduce, pp_grad "
                         "with the summed coefficients); autograd: energy forward + adjoint backward; "
                         "block-adjoint: per-block energies forward + vector-output adjoint; "
                         "binned: the binned fast scheme (terms counted as N Mx My); "
                         "place: one iteration of the Sec. IV placement loop (density, LSE "
                         "wirelength, Nesterov step, overflow) on a synthetic netlist")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
