"""Python binding of the C ABI (include/pp.h): argument marshalling only.

torch provides device memory and the current stream; every arithmetic step of
the evaluation runs in the CUDA library.  There is no fallback: if libpp.so is
missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional

import numpy as np
import torch

from . import build_lib

PRECISIONS = {"fp32": 0, "tf32": 1, "bf16x3": 2}
SAMPLES = {"rect": 0, "center": 1}
STATUS = {0: "PP_OK", 1: "PP_EINVAL", 2: "PP_ENOMEM_WS", 3: "PP_ECUDA", 4: "PP_ETIMEOUT",
          5: "PP_ENOTSUP"}
# Normalised max-error bounds used by the parity tests (max |err| / max |ref|).
TOLERANCE = {"fp32": 1e-6, "tf32": 1e-3, "bf16x3": 1e-4}

Precision = PRECISIONS
Sample = SAMPLES


class PPError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Problem(ctypes.Structure):
    _fields_ = [("W", ctypes.c_double), ("H", ctypes.c_double), ("n", ctypes.c_int64),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("h", ctypes.c_void_p), ("c", ctypes.c_void_p),
                ("Mx", ctypes.c_int32), ("My", ctypes.c_int32)]


class Netlist(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int32), ("n_nets", ctypes.c_int32),
                ("net_ptr", ctypes.c_void_p), ("net_pin", ctypes.c_void_p),
                ("cell_ptr", ctypes.c_void_p), ("cell_net", ctypes.c_void_p)]


class PlaceIterationArgs(ctypes.Structure):
    """pp_place_iteration_args (one placement-loop iteration in one call)."""
    _fields_ = [("netlist", ctypes.POINTER(Netlist)), ("W", ctypes.c_double), ("H", ctypes.c_double),
                ("M", ctypes.c_int32), ("density", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("n_overflow", ctypes.c_int64)] + \
              [(k, ctypes.c_void_p) for k in ("w", "h", "c", "q", "movable", "ux", "uy", "vx", "vy",
                                              "vpx", "vpy", "gpx", "gpy")] + \
              [(k, ctypes.c_float) for k in ("lam", "gamma", "alpha0", "coef", "target")] + \
              [("stats", ctypes.c_void_p), ("scalars", ctypes.c_void_p)]


class PlaceSchedule(ctypes.Structure):
    """pp_place_schedule (the loop's stop rule and the constants of its scalar update)."""
    _fields_ = [("max_iters", ctypes.c_int32), ("reserved", ctypes.c_int32), ("tau_stop", ctypes.c_double),
                ("bin_area", ctypes.c_double), ("area_mov", ctypes.c_double), ("bin_w", ctypes.c_double)]


class PlaceState(ctypes.Structure):
    """pp_place_state (the loop's scalars between iterations; lives on the device)."""
    _fields_ = [("lam", ctypes.c_double), ("gamma", ctypes.c_double), ("a_k", ctypes.c_double),
                ("hpwl_prev", ctypes.c_double), ("d_ref", ctypes.c_double), ("tau", ctypes.c_double),
                ("k", ctypes.c_int64), ("stop", ctypes.c_int32), ("run_count", ctypes.c_int32),
                ("scalars", ctypes.c_float * 4)]


class PlaceRecord(ctypes.Structure):
    """pp_place_record (one iteration of a device-resident run)."""
    _fields_ = [("k", ctypes.c_int64), ("stop", ctypes.c_int32), ("reserved", ctypes.c_int32)] + \
               [(f, ctypes.c_double) for f in ("tau", "w_lse", "hpwl", "e", "lam", "gamma")]


PLACE_STOP = {0: "running", 1: "converged", 2: "max_iters", 3: "nonfinite", 4: "device_error", 5: "bad_state"}

_LIB = None
EXPORTS = ("pp_workspace_size", "pp_coeffs", "pp_energy", "pp_grad", "pp_sync_status",
           "pp_last_error", "pp_version", "pp_timing_enable", "pp_timing_collect",
           "pp_grad_noalloc", "pp_phase_eval", "pp_binned_workspace_size", "pp_binned_grad",
           "pp_energy_from_coeffs", "pp_descent_step",
           "pp_wirelength_workspace_size", "pp_wirelength", "pp_place_combine", "pp_step_norms",
           "pp_nesterov_step", "pp_overflow", "pp_place_workspace_size", "pp_place_iteration",
           "pp_check_wait_timeout", "pp_grad_adjoint", "pp_coeffs_accumulate",
           "pp_grad_host_workspace_size", "pp_grad_host", "pp_place_run")


def lib_path() -> str:
    return build_lib.LIB


def lib() -> ctypes.CDLL:
    """Load libpp.so (built in-tree by __graft_entry__.build())."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(build_lib.LIB):
            raise RuntimeError(f"{build_lib.LIB} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(build_lib.LIB)
        P = ctypes.POINTER(Problem)
        vp, sz, i = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
        L.pp_workspace_size.argtypes = [P, i]
        L.pp_workspace_size.restype = sz
        L.pp_coeffs.argtypes = [P, i, vp, vp, sz, vp]
        L.pp_coeffs.restype = i
        L.pp_energy.argtypes = [P, i, i, vp, vp, vp, vp, sz, vp]
        L.pp_energy.restype = i
        L.pp_grad.argtypes = [P, i, i, vp, vp, vp, vp, vp, vp, sz, vp]
        L.pp_grad.restype = i
        L.pp_sync_status.argtypes = [vp]
        L.pp_sync_status.restype = i
        L.pp_phase_eval.argtypes = [vp, ctypes.c_double, vp, ctypes.c_int64, i, vp, vp]
        L.pp_phase_eval.restype = i
        L.pp_binned_workspace_size.argtypes = [P, ctypes.c_int32]
        L.pp_binned_workspace_size.restype = sz
        L.pp_binned_grad.argtypes = [P, i, ctypes.c_int32, vp, vp, vp, vp, vp, vp, sz, vp]
        L.pp_binned_grad.restype = i
        L.pp_energy_from_coeffs.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                            ctypes.c_double, vp, vp]
        L.pp_energy_from_coeffs.restype = i
        L.pp_descent_step.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int64, vp, vp, vp,
                                      vp, vp, vp, vp, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_uint64, ctypes.c_uint64, vp]
        L.pp_descent_step.restype = i
        NL = ctypes.POINTER(Netlist)
        f32, i64 = ctypes.c_float, ctypes.c_int64
        L.pp_wirelength_workspace_size.argtypes = [ctypes.c_int32]
        L.pp_wirelength_workspace_size.restype = sz
        L.pp_wirelength.argtypes = [NL, vp, vp, f32, vp, vp, vp, vp, sz, vp]
        L.pp_wirelength.restype = i
        L.pp_place_combine.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, f32, vp, vp, vp]
        L.pp_place_combine.restype = i
        L.pp_step_norms.argtypes = [i64] + [vp] * 9 + [vp]
        L.pp_step_norms.restype = i
        L.pp_nesterov_step.argtypes = ([i64, ctypes.c_double, ctypes.c_double] + [vp] * 14 +
                                       [f32, f32, vp])
        L.pp_nesterov_step.restype = i
        L.pp_overflow.argtypes = [P, ctypes.c_int32, f32, vp, vp, vp]
        L.pp_overflow.restype = i
        PA = ctypes.POINTER(PlaceIterationArgs)
        L.pp_place_workspace_size.argtypes = [PA]
        L.pp_place_workspace_size.restype = sz
        L.pp_place_iteration.argtypes = [PA, vp, sz, vp]
        L.pp_place_iteration.restype = i
        L.pp_place_run.argtypes = [PA, ctypes.POINTER(PlaceSchedule), vp, vp, vp, sz, vp]
        L.pp_place_run.restype = i
        L.pp_check_wait_timeout.argtypes = [ctypes.c_uint64, vp]
        L.pp_check_wait_timeout.restype = i
        L.pp_last_error.argtypes = []
        L.pp_last_error.restype = ctypes.c_char_p
        L.pp_version.argtypes = []
        L.pp_version.restype = ctypes.c_char_p
        L.pp_grad_adjoint.argtypes = [P, i, i, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        L.pp_grad_adjoint.restype = i
        L.pp_coeffs_accumulate.argtypes = [P, i, vp, vp, vp, sz, vp]
        L.pp_coeffs_accumulate.restype = i
        L.pp_grad_host_workspace_size.argtypes = [P, i]
        L.pp_grad_host_workspace_size.restype = sz
        L.pp_grad_host.argtypes = [P, i, i, vp, vp, vp, vp, vp, sz, vp]
        L.pp_grad_host.restype = i
        L.pp_grad_noalloc.argtypes = [P, i, vp, vp, vp, vp, vp]
        L.pp_grad_noalloc.restype = i
        L.pp_timing_enable.argtypes = [i]
        L.pp_timing_enable.restype = None
        L.pp_timing_collect.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
        L.pp_timing_collect.restype = i
        _LIB = L
    return _LIB


KERNELS = ("prep", "coeff", "finish", "energy")


def timing_enable(on: bool = True):
    lib().pp_timing_enable(1 if on else 0)


def timing_collect():
    """{kernel: (launches, summed device ms)} since the previous collect."""
    n = (ctypes.c_int64 * 4)()
    ms = (ctypes.c_double * 4)()
    _check(lib().pp_timing_collect(n, ms))
    return {k: (int(n[i]), float(ms[i])) for i, k in enumerate(KERNELS)}


def version() -> str:
    return lib().pp_version().decode()


def available_precisions():
    v = version()
    return ("fp32", "tf32", "bf16x3") if "tcgen05" in v else ("fp32",)


def _check(st: int):
    if st != 0:
        raise PPError(st, lib().pp_last_error().decode())


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream_handle(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def make_problem(x, y, w, h, c, W, H, Mx, My) -> Problem:
    n = x.numel()
    for name, t in (("x", x), ("y", y), ("w", w), ("h", h), ("c", c)):
        if t is None:
            continue
        if t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"{name} must be a contiguous float32 tensor of {n} elements")
        if t.device != x.device or t.device.type != "cuda":
            raise ValueError(f"{name} must be a CUDA tensor on {x.device}")
    return Problem(float(W), float(H), n, _ptr(x) if n else None, _ptr(y) if n else None,
                   _ptr(w) if n else None, _ptr(h) if n else None,
                   _ptr(c) if (c is not None and n) else None, int(Mx), int(My))


_WS = {}


def workspace(prob: Problem, prec: str, device) -> torch.Tensor:
    """A cached device workspace of at least pp_workspace_size() bytes."""
    need = lib().pp_workspace_size(ctypes.byref(prob), PRECISIONS[prec])
    if need == 0:
        _check(1)
    key = (torch.device(device).index, torch.cuda.current_stream(device).cuda_stream)
    buf = _WS.get(key)
    if buf is None or buf.numel() < need:
        buf = torch.empty(need, dtype=torch.uint8, device=device)
        _WS[key] = buf
    return buf


def coeffs(x, y, w, h, c, W, H, Mx, My, prec="fp32", out=None):
    """pp_coeffs: the Mx x My coefficient matrix a (float32, u-major)."""
    prob = make_problem(x, y, w, h, c, W, H, Mx, My)
    dev = x.device
    a = out if out is not None else torch.empty((Mx, My), dtype=torch.float32, device=dev)
    ws = workspace(prob, prec, dev)
    _check(lib().pp_coeffs(ctypes.byref(prob), PRECISIONS[prec], a.data_ptr(), ws.data_ptr(),
                           ws.numel(), _stream_handle(dev)))
    return a


def energy(x, y, w, h, c, W, H, Mx, My, prec="fp32", sample="rect", a=None,
           want_block=True):
    """pp_energy: (N_i per block or None, E as a 1-element float64 tensor)."""
    prob = make_problem(x, y, w, h, c, W, H, Mx, My)
    dev = x.device
    n = x.numel()
    eb = torch.empty(n, dtype=torch.float32, device=dev) if want_block else None
    et = torch.empty(1, dtype=torch.float64, device=dev)
    ws = workspace(prob, prec, dev)
    _check(lib().pp_energy(ctypes.byref(prob), PRECISIONS[prec], SAMPLES[sample], _ptr(a),
                           _ptr(eb) if n else None, et.data_ptr(), ws.data_ptr(), ws.numel(),
                           _stream_handle(dev)))
    return eb, et


def grad(x, y, w, h, c, W, H, Mx, My, prec="fp32", sample="rect", a=None, want_energy=True,
         out=None):
    """pp_grad: (gx, gy, N_i or None, E or None)."""
    prob = make_problem(x, y, w, h, c, W, H, Mx, My)
    dev = x.device
    n = x.numel()
    if out is None:
        gx = torch.empty(n, dtype=torch.float32, device=dev)
        gy = torch.empty(n, dtype=torch.float32, device=dev)
        eb = torch.empty(n, dtype=torch.float32, device=dev) if want_energy else None
        et = torch.empty(1, dtype=torch.float64, device=dev) if want_energy else None
    else:
        gx, gy, eb, et = out
    ws = workspace(prob, prec, dev)
    _check(lib().pp_grad(ctypes.byref(prob), PRECISIONS[prec], SAMPLES[sample], _ptr(a),
                         _ptr(gx) if n else None, _ptr(gy) if n else None,
                         _ptr(eb) if (eb is not None and n) else None, _ptr(et),
                         ws.data_ptr(), ws.numel(), _stream_handle(dev)))
    return gx, gy, eb, et


_WS_HOST = {}


def grad_host(x, y, w, h, c, W, H, Mx, My, prec="fp32", sample="rect", out=None, device=None):
    """pp_grad_host: the evaluation of `grad` for a placement in host memory, the
    results written to host memory.  x, y, w, h, c (c may be None): contiguous
    float32 CPU tensors of n; out: (gx, gy, N_i, E) CPU tensors (float32 n x3,
    float64 1), allocated pinned when None.  Pinned tensors are read and written in
    place by the kernels; pageable ones are staged.  Asynchronous on the current
    stream of `device` (default: the current CUDA device): synchronize it before
    reading the outputs."""
    n = x.numel()
    for name, t in (("x", x), ("y", y), ("w", w), ("h", h), ("c", c)):
        if t is None:
            continue
        if t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != n or t.device.type != "cpu":
            raise ValueError(f"{name} must be a contiguous float32 CPU tensor of {n} elements")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    prob = Problem(float(W), float(H), n, _ptr(x) if n else None, _ptr(y) if n else None,
                   _ptr(w) if n else None, _ptr(h) if n else None,
                   _ptr(c) if (c is not None and n) else None, int(Mx), int(My))
    if out is None:
        out = (torch.empty(n, dtype=torch.float32).pin_memory(), torch.empty(n, dtype=torch.float32).pin_memory(),
               torch.empty(n, dtype=torch.float32).pin_memory(), torch.empty(1, dtype=torch.float64).pin_memory())
    gx, gy, eb, et = out
    need = lib().pp_grad_host_workspace_size(ctypes.byref(prob), PRECISIONS[prec])
    if need == 0:
        _check(1)
    key = (dev.index, torch.cuda.current_stream(dev).cuda_stream)
    ws = _WS_HOST.get(key)
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
        _WS_HOST[key] = ws
    _check(lib().pp_grad_host(ctypes.byref(prob), PRECISIONS[prec], SAMPLES[sample],
                              _ptr(gx) if n else None, _ptr(gy) if n else None,
                              _ptr(eb) if (eb is not None and n) else None, _ptr(et),
                              ws.data_ptr(), ws.numel(), _stream_handle(dev)))
    return gx, gy, eb, et


def _mask(movable, n, device):
    if movable is None:
        return None
    m = movable if movable.dtype == torch.uint8 else movable.to(torch.uint8)
    m = m.contiguous()
    if m.numel() != n or m.device != torch.device(device):
        raise ValueError(f"movable must be a bool/uint8 tensor of {n} elements on {device}")
    return m


def grad_adjoint(x, y, w, h, c, W, H, Mx, My, prec="fp32", sample="rect", g_total=None, g_block=None,
                 movable=None, want_energy=False):
    """pp_grad_adjoint: (dL/dx, dL/dy, N_i or None, E or None) for
    L = g_total * E + sum_i g_block_i N_i; g_total a 1-element float64 device tensor
    (or None), g_block a float32 device tensor of n (or None); blocks whose `movable`
    entry is False get 0."""
    prob = make_problem(x, y, w, h, c, W, H, Mx, My)
    dev = x.device
    n = x.numel()
    if g_total is not None:
        g_total = g_total.reshape(1)
        if g_total.dtype != torch.float64:
            g_total = g_total.to(torch.float64)
        g_total = g_total.contiguous()
    if g_block is not None:
        g_block = g_block.contiguous()
        if g_block.dtype != torch.float32 or g_block.numel() != n:
            raise ValueError(f"g_block must be a float32 tensor of {n} elements")
    mv = _mask(movable, n, dev)
    gx = torch.empty(n, dtype=torch.float32, device=dev)
    gy = torch.empty(n, dtype=torch.float32, device=dev)
    eb = torch.empty(n, dtype=torch.float32, device=dev) if want_energy else None
    et = torch.empty(1, dtype=torch.float64, device=dev) if want_energy else None
    ws = workspace(prob, prec, dev)
    _check(lib().pp_grad_adjoint(ctypes.byref(prob), PRECISIONS[prec], SAMPLES[sample], _ptr(g_total),
                                 _ptr(g_block) if n else None, _ptr(mv) if n else None,
                                 _ptr(gx) if n else None, _ptr(gy) if n else None,
                                 _ptr(eb) if (eb is not None and n) else None, _ptr(et),
                                 ws.data_ptr(), ws.numel(), _stream_handle(dev)))
    return gx, gy, eb, et


def coeffs_accumulate(x, y, w, h, c, W, H, Mx, My, a64, prec="fp32", a_out=None):
    """pp_coeffs_accumulate: a64 (float64 Mx x My device tensor) += the coefficients of
    these blocks; a_out (optional float32 Mx x My) receives the rounded running sum.
    With zero blocks only a_out is written."""
    prob = make_problem(x, y, w, h, c, W, H, Mx, My)
    dev = a64.device
    if a64.dtype != torch.float64 or not a64.is_contiguous() or a64.numel() != Mx * My:
        raise ValueError("a64 must be a contiguous float64 tensor of Mx * My elements")
    if a_out is not None and (a_out.dtype != torch.float32 or not a_out.is_contiguous()
                              or a_out.numel() != Mx * My):
        raise ValueError("a_out must be a contiguous float32 tensor of Mx * My elements")
    ws = workspace(prob, prec, dev)
    _check(lib().pp_coeffs_accumulate(ctypes.byref(prob), PRECISIONS[prec], _ptr(a64), _ptr(a_out),
                                      ws.data_ptr(), ws.numel(), _stream_handle(dev)))
    return a64


def grad_noalloc(x, y, w, h, c, W, H, Mx, My, sample="rect", out=None):
    """pp_grad_noalloc: the FP32 evaluation with the library's static scratch instead
    of a workspace (for callers that cannot allocate).  Returns (gx, gy, N_i, E)."""
    prob = make_problem(x, y, w, h, c, W, H, Mx, My)
    dev = x.device
    n = x.numel()
    if out is None:
        out = (torch.empty(n, dtype=torch.float32, device=dev),
               torch.empty(n, dtype=torch.float32, device=dev),
               torch.empty(n, dtype=torch.float32, device=dev),
               torch.empty(1, dtype=torch.float64, device=dev))
    gx, gy, eb, et = out
    _check(lib().pp_grad_noalloc(ctypes.byref(prob), SAMPLES[sample], _ptr(gx) if n else None,
                                 _ptr(gy) if n else None, _ptr(eb) if (eb is not None and n) else None,
                                 _ptr(et), _stream_handle(dev)))
    return gx, gy, eb, et


def sync_status(device=None):
    """pp_sync_status on the current stream: raises PPError if a kernel timed out."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    _check(lib().pp_sync_status(_stream_handle(dev)))


def phase_eval(x, L: float, m, evaluator: int = 0):
    """pp_phase_eval: (cos, sin)(pi * (m * x / L mod 2)) per element, shape (count, 2);
    x float32 and m int32 device tensors of equal length."""
    x = x.contiguous()
    m = m.contiguous()
    if x.dtype != torch.float32 or m.dtype != torch.int32 or x.numel() != m.numel():
        raise ValueError("x must be float32 and m int32, of equal length")
    out = torch.empty((x.numel(), 2), dtype=torch.float32, device=x.device)
    _check(lib().pp_phase_eval(_ptr(x), float(L), _ptr(m), x.numel(), int(evaluator), _ptr(out),
                               _stream_handle(x.device)))
    return out


def binned_grad(x, y, w, h, c, W, H, Mx, My, m, prec="fp32", want_coeffs=True):
    """pp_binned_grad, the binned fast scheme on m x m bins: (gx, gy, N_i, E, a or None)."""
    prob = make_problem(x, y, w, h, c, W, H, Mx, My)
    dev = x.device
    n = x.numel()
    need = lib().pp_binned_workspace_size(ctypes.byref(prob), int(m))
    if need == 0:
        raise PPError(1, lib().pp_last_error().decode())
    ws = torch.empty(need + 256, dtype=torch.uint8, device=dev)
    base = (ws.data_ptr() + 255) // 256 * 256
    gx = torch.empty(n, dtype=torch.float32, device=dev)
    gy = torch.empty(n, dtype=torch.float32, device=dev)
    eb = torch.empty(n, dtype=torch.float32, device=dev)
    et = torch.empty(1, dtype=torch.float64, device=dev)
    a = torch.empty((Mx, My), dtype=torch.float32, device=dev) if want_coeffs else None
    _check(lib().pp_binned_grad(ctypes.byref(prob), PRECISIONS[prec], int(m), _ptr(a),
                                _ptr(gx) if n else None, _ptr(gy) if n else None, _ptr(eb) if n else None,
                                _ptr(et), base, need, _stream_handle(dev)))
    return gx, gy, eb, et, a


def energy_from_coeffs(a, W, H):
    """pp_energy_from_coeffs: E = 1/2 sum a^2 / G (FP64) of an Mx x My float32 device tensor."""
    a = a.contiguous()
    if a.dtype != torch.float32 or a.dim() != 2:
        raise ValueError("a must be a 2-D float32 tensor")
    e = torch.empty(1, dtype=torch.float64, device=a.device)
    _check(lib().pp_energy_from_coeffs(_ptr(a), a.shape[0], a.shape[1], float(W), float(H), _ptr(e),
                                       _stream_handle(a.device)))
    return e


def descent_step(x, y, w, h, gx, gy, W, H, lr, sigma, seed, step, movable=None):
    """pp_descent_step: in-place position update of float32 device tensors x, y
    (movable: optional bool/uint8 device mask)."""
    for t in (x, y, w, h, gx, gy):
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError("descent_step takes contiguous float32 tensors")
    mv = None if movable is None else movable.to(torch.uint8).contiguous()
    _check(lib().pp_descent_step(float(W), float(H), x.numel(), _ptr(x), _ptr(y), _ptr(w), _ptr(h),
                                 _ptr(gx), _ptr(gy), _ptr(mv), float(lr), float(sigma),
                                 int(seed) & (2 ** 64 - 1), int(step), _stream_handle(x.device)))


def check_wait_timeout(limit_ns: int, device=None):
    """pp_check_wait_timeout on the current stream: one kernel whose bounded wait
    runs out after `limit_ns`; the following sync_status() raises PP_ETIMEOUT."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    _check(lib().pp_check_wait_timeout(int(limit_ns), _stream_handle(dev)))


def to_device(p, device):
    """Upload a synth.Placement's arrays to `device`."""
    t = lambda a: None if a is None else torch.from_numpy(a).to(device)
    return t(p.x), t(p.y), t(p.w), t(p.h), t(p.c)


def evaluate(p, prec="fp32", device="cuda", sample="rect"):
    """Coefficients (pp_coeffs) and a full energy + gradient evaluation (pp_grad with
    a = NULL) of a synth.Placement; results as torch tensors plus E as a float."""
    x, y, w, h, c = to_device(p, device)
    a = coeffs(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec)
    gx, gy, eb, et = grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec, sample)
    sync_status(device)
    return dict(a=a, N=eb, gx=gx, gy=gy, E=float(et.item()))


class PoissonEnergy(torch.autograd.Function):
    """E = 1/2 sum_i N_i as a differentiable function of the block centres.

    forward:  pp_energy (coefficients computed inside the call, not kept)
    backward: pp_grad_adjoint with g_total = the upstream gradient: the coefficients
              are recomputed rather than stored, and the library scales dE/dx, dE/dy
              by it.  Blocks whose `movable` entry is False receive zero gradient.
    """

    @staticmethod
    def forward(ctx, x, y, w, h, c, W, H, Mx, My, prec="fp32", sample="rect", movable=None):
        _, et = energy(x, y, w, h, c, W, H, Mx, My, prec, sample, want_block=False)
        ctx.save_for_backward(x, y, w, h, c if c is not None else torch.empty(0, device=x.device),
                              movable if movable is not None else torch.empty(0, device=x.device))
        ctx.args = (W, H, Mx, My, prec, sample, c is not None, movable is not None)
        return et[0]

    @staticmethod
    def backward(ctx, g):
        x, y, w, h, c, mov = ctx.saved_tensors
        W, H, Mx, My, prec, sample, has_c, has_mov = ctx.args
        gx, gy, _, _ = grad_adjoint(x.detach(), y.detach(), w, h, c if has_c else None, W, H, Mx, My,
                                    prec, sample, g_total=g, movable=mov if has_mov else None)
        return (gx if ctx.needs_input_grad[0] else None,
                gy if ctx.needs_input_grad[1] else None,
                None, None, None, None, None, None, None, None, None, None)


class PoissonBlockEnergies(torch.autograd.Function):
    """The per-block energies N_i (rectangle reading) as a differentiable function of
    the block centres, for any upstream gradient g.

    With L = sum_i g_i N_i, N_i = sum_uv X_iu a_uv Y_iv and a = G o S(x, y):
      dL/dx_j = g_j h_j + h^b_j,
    where h_j = sum_uv X'_ju a_uv Y_jv is the gradient pp_grad returns with the
    placement's own coefficients a, and h^b_j the same with b = G o sum_i g_i X_i Y_i^T,
    i.e. the coefficients of the same blocks with charges c_i g_i.  For g = 1/2
    everywhere b = a/2 and dL/dx = h = dE/dx.  The backward is one library call,
    pp_grad_adjoint with g_block = g: it recomputes a, computes b and combines the
    two energy passes on the device (two coefficient and two energy contractions).
    Blocks whose `movable` entry is False receive zero gradient.
    """

    @staticmethod
    def forward(ctx, x, y, w, h, c, W, H, Mx, My, prec="fp32", movable=None):
        eb, _ = energy(x, y, w, h, c, W, H, Mx, My, prec, "rect")
        ctx.save_for_backward(x, y, w, h, c if c is not None else torch.empty(0, device=x.device),
                              movable if movable is not None else torch.empty(0, device=x.device))
        ctx.args = (W, H, Mx, My, prec, c is not None, movable is not None)
        return eb

    @staticmethod
    def backward(ctx, g):
        x, y, w, h, c, mov = ctx.saved_tensors
        W, H, Mx, My, prec, has_c, has_mov = ctx.args
        gx, gy, _, _ = grad_adjoint(x.detach(), y.detach(), w, h, c if has_c else None, W, H, Mx, My,
                                    prec, "rect", g_block=g.to(torch.float32),
                                    movable=mov if has_mov else None)
        return (gx if ctx.needs_input_grad[0] else None,
                gy if ctx.needs_input_grad[1] else None,
                None, None, None, None, None, None, None, None, None)


# ---- placement loop (Sec. IV) ---------------------------------------------------

class DeviceNetlist:
    """A netlist in both orientations on the device (int32 CSR arrays) and its
    C-ABI view; built from host arrays (net_ptr, net_pin) once per netlist."""

    def __init__(self, n_cells: int, net_ptr, net_pin, device="cuda"):
        net_ptr = np.asarray(net_ptr, dtype=np.int64)
        net_pin = np.asarray(net_pin, dtype=np.int64)
        n_nets = len(net_ptr) - 1
        # the kernels index with these arrays: check them here, once
        if n_nets < 0 or net_ptr[0] != 0 or np.any(np.diff(net_ptr) < 0) or net_ptr[-1] != len(net_pin):
            raise ValueError("net_ptr must start at 0, not decrease and end at len(net_pin)")
        if len(net_pin) and (net_pin.min() < 0 or net_pin.max() >= n_cells):
            raise ValueError("net_pin entries must lie in [0, n_cells)")
        if n_cells > 2**31 - 1 or len(net_pin) > 2**31 - 1:
            raise ValueError("netlist too large for int32 indices")
        # the transpose: cell -> its nets, nets in increasing order per cell
        net_of_pin = np.repeat(np.arange(n_nets, dtype=np.int64), np.diff(net_ptr))
        order = np.lexsort((net_of_pin, net_pin))
        cell_ptr = np.zeros(n_cells + 1, dtype=np.int64)
        np.add.at(cell_ptr, net_pin + 1, 1)
        cell_ptr = np.cumsum(cell_ptr)
        dev = torch.device(device)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).to(dev)
        self.n_cells, self.n_nets = int(n_cells), int(n_nets)
        self.net_ptr, self.net_pin = t(net_ptr), t(net_pin)
        self.cell_ptr, self.cell_net = t(cell_ptr), t(net_of_pin[order])
        self.c = Netlist(self.n_cells, self.n_nets, _ptr(self.net_ptr), _ptr(self.net_pin),
                         _ptr(self.cell_ptr), _ptr(self.cell_net))
        self.ws = torch.empty(lib().pp_wirelength_workspace_size(self.n_nets), dtype=torch.uint8,
                              device=dev)

    def degree(self) -> torch.Tensor:
        return (self.cell_ptr[1:] - self.cell_ptr[:-1]).float()


def wirelength(nl: DeviceNetlist, x, y, gamma: float, out=None):
    """pp_wirelength: (gx, gy, out) with out = device double [W_LSE, HPWL]."""
    gx = torch.empty_like(x)
    gy = torch.empty_like(y)
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device=x.device)
    _check(lib().pp_wirelength(ctypes.byref(nl.c), _ptr(x), _ptr(y), float(gamma), _ptr(gx), _ptr(gy),
                               _ptr(out), _ptr(nl.ws), nl.ws.numel(), _stream_handle(x.device)))
    return gx, gy, out


def place_combine(gwx, gwy, gnx, gny, cell_ptr, q, movable, lam: float):
    gx = torch.empty_like(gwx)
    gy = torch.empty_like(gwy)
    _check(lib().pp_place_combine(gwx.numel(), _ptr(gwx), _ptr(gwy), _ptr(gnx), _ptr(gny), _ptr(cell_ptr),
                                  _ptr(q), _ptr(movable), float(lam), _ptr(gx), _ptr(gy),
                                  _stream_handle(gwx.device)))
    return gx, gy


def step_norms(vx, vy, vpx, vpy, gx, gy, gpx, gpy, norms):
    _check(lib().pp_step_norms(vx.numel(), _ptr(vx), _ptr(vy), _ptr(vpx), _ptr(vpy), _ptr(gx), _ptr(gy),
                               _ptr(gpx), _ptr(gpy), _ptr(norms), _stream_handle(vx.device)))
    return norms


def nesterov_step(W, H, ux, uy, vx, vy, vpx, vpy, gx, gy, gpx, gpy, w, h, movable, norms, alpha0, coef):
    """pp_nesterov_step, in place on u, v, vp, gp."""
    _check(lib().pp_nesterov_step(ux.numel(), float(W), float(H), _ptr(ux), _ptr(uy), _ptr(vx), _ptr(vy),
                                  _ptr(vpx), _ptr(vpy), _ptr(gx), _ptr(gy), _ptr(gpx), _ptr(gpy), _ptr(w),
                                  _ptr(h), _ptr(movable), _ptr(norms), float(alpha0), float(coef),
                                  _stream_handle(ux.device)))


DENSITIES = {"exact": 0, "binned": 1}


class PlaceIteration:
    """pp_place_iteration bound to one placement state: the C-ABI argument block,
    its workspace and the 4-double stats buffer {overflow excess, W_LSE, HPWL, E}.
    The tensors are referenced, not copied: the call updates u, v, vp, gp in place.

    graph=True: the scalars live in a device array the kernels read as they run, the
    call is captured once in a CUDA graph, and every later call writes the four
    scalars to the device and replays the graph (no per-call argument checks or
    launches on the host).  The captured call keeps the workspace, state and stats
    pointers, so none of those tensors may be reallocated."""

    def __init__(self, nl: DeviceNetlist, W, H, M: int, density: str, prec: str, n_overflow: int,
                 w, h, c, q, movable, ux, uy, vx, vy, vpx, vpy, gpx, gpy, target: float = 1.0,
                 graph: bool = False):
        self.nl = nl
        self.keep = (w, h, c, q, movable, ux, uy, vx, vy, vpx, vpy, gpx, gpy)
        dev = ux.device
        self.stats = torch.zeros(4, dtype=torch.float64, device=dev)
        self.a = PlaceIterationArgs(ctypes.pointer(nl.c), float(W), float(H), int(M), DENSITIES[density],
                                    PRECISIONS[prec], 0, int(n_overflow),
                                    *[_ptr(t) for t in self.keep], 0.0, 1.0, 0.0, 0.0, float(target),
                                    _ptr(self.stats), None)
        nbytes = lib().pp_place_workspace_size(ctypes.byref(self.a))
        if nbytes == 0:
            raise PPError(1, lib().pp_last_error().decode())
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.graph, self.graph_error, self.scal_dev = None, None, None
        if graph:
            self.scal_dev = torch.zeros(4, dtype=torch.float32, device=dev)
            self.a.scalars = _ptr(self.scal_dev)

    def _call(self):
        _check(lib().pp_place_iteration(ctypes.byref(self.a), _ptr(self.ws), self.ws.numel(),
                                        _stream_handle(self.ws.device)))

    def __call__(self, lam: float, gamma: float, coef: float, alpha0: float = 0.0):
        a = self.a
        a.lam, a.gamma, a.coef, a.alpha0 = float(lam), float(gamma), float(coef), float(alpha0)
        if self.scal_dev is None:
            self._call()
            return self.stats
        if not (math.isfinite(lam) and lam >= 0 and math.isfinite(gamma) and gamma > 0
                and math.isfinite(alpha0) and alpha0 >= 0 and math.isfinite(coef)):
            raise PPError(1, "lambda, gamma, alpha0 must be finite (lambda, alpha0 >= 0, gamma > 0), coef finite")
        dev = self.ws.device
        if self.graph is None:          # capture once (nothing runs during the capture)
            g = torch.cuda.CUDAGraph()
            main = torch.cuda.current_stream(dev)
            side = torch.cuda.Stream(device=dev)
            side.wait_stream(main)
            try:
                with torch.cuda.graph(g, stream=side):
                    self._call()
            except Exception as e:      # keep the eager call (same kernels) and say why
                torch.cuda.set_stream(main)
                self.graph_error = f"{type(e).__name__}: {e}"
                self.a.scalars = None
                self.scal_dev = None
                main.wait_stream(side)
                self._call()
                return self.stats
            main.wait_stream(side)
            self.graph = g
        # a pinned staging tensor per call: the host allocator keeps it until the copy is done
        src = torch.tensor([lam, gamma, alpha0, coef], dtype=torch.float32).pin_memory()
        self.scal_dev.copy_(src, non_blocking=True)
        self.graph.replay()
        return self.stats

    def run(self, state: PlaceState, sched: PlaceSchedule):
        """pp_place_run: iterations state.k, state.k + 1, ... on the device until a stop
        condition holds.  Returns (the state after the run, the records made, in order).
        One graph launch; the host waits for it once, at the end."""
        dev = self.ws.device
        st_dev = torch.frombuffer(bytearray(bytes(state)), dtype=torch.uint8).to(dev)
        k0 = int(state.k)
        trace = torch.zeros((max(int(sched.max_iters), 1), ctypes.sizeof(PlaceRecord)), dtype=torch.uint8,
                            device=dev)
        _check(lib().pp_place_run(ctypes.byref(self.a), ctypes.byref(sched), _ptr(st_dev), _ptr(trace), _ptr(self.ws),
                                  self.ws.numel(), _stream_handle(dev)))
        out = PlaceState.from_buffer_copy(bytes(st_dev.cpu().numpy()))
        k1 = min(int(out.k), int(sched.max_iters))
        raw = bytes(trace[k0:k1].cpu().numpy()) if k1 > k0 else b""
        sz = ctypes.sizeof(PlaceRecord)
        recs = [PlaceRecord.from_buffer_copy(raw[i * sz:(i + 1) * sz]) for i in range(k1 - k0)]
        return out, recs


def overflow(x, y, w, h, W, H, m: int, target: float = 1.0, bins=None, out=None):
    """pp_overflow: (excess in bin areas as a device double, bin density m x m)."""
    if bins is None:
        bins = torch.empty((m, m), dtype=torch.float32, device=x.device)
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=x.device)
    prob = make_problem(x, y, w, h, None, W, H, 1, 1)
    _check(lib().pp_overflow(ctypes.byref(prob), int(m), float(target), _ptr(bins), _ptr(out),
                             _stream_handle(x.device)))
    return out, bins
