"""The allocation-free entry point pp_grad_noalloc, called through the C ABI.

It serves callers that cannot allocate device memory when they evaluate the
energy; its scratch is a static device array inside the library.  Its outputs
must equal those of pp_grad (FP32, coefficients computed in the call) within the
FP32 parity tolerance, on two calls in a row -- the second with a different
problem, so leftovers of the first call in the shared scratch would show -- and
at the largest problem its scratch holds they must also match the FP64 oracle.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import series as O
from paper_2307_12041_gb300 import synth

pytestmark = pytest.mark.gpu

MAX_BLOCKS = 32768      # PP_STATIC_MAX_BLOCKS
MAX_MODES = 256         # PP_STATIC_MAX_MODES


def _close(a, b, tol):
    scale = float(b.abs().max())
    return float((a - b).abs().max()) <= tol * max(scale, 1e-30)


@pytest.mark.parametrize("sample", ["rect", "center"])
def test_noalloc_matches_workspace_entry_point_twice(pp, sample):
    B = pp.binding
    tol = B.TOLERANCE["fp32"]
    dev = torch.device("cuda")
    cases = [synth.uniform_blocks(3001, 96, 80, seed=21, W=1.3, H=0.8, charge=True),
             synth.cell_mix(1200, 200, 256, seed=22)]
    for p in cases:
        x, y, w, h, c = B.to_device(p, dev)
        ref = B.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, "fp32", sample)
        got = B.grad_noalloc(x, y, w, h, c, p.W, p.H, p.Mx, p.My, sample)
        B.sync_status(dev)
        for r, g in zip(ref, got):
            assert _close(g, r, tol)
        assert abs(float(got[3]) - float(ref[3])) <= tol * abs(float(ref[3]))


def test_noalloc_at_its_limits_matches_pp_grad_and_the_oracle(pp):
    """n = PP_STATIC_MAX_BLOCKS and Mx = My = PP_STATIC_MAX_MODES fill every region of
    the static scratch (both record regions, the FP64 sums and the operand) to its
    end; then a small problem, which must not see the large one's leftovers."""
    B = pp.binding
    tol = B.TOLERANCE["fp32"]
    dev = torch.device("cuda")
    big = synth.cell_mix(MAX_BLOCKS, MAX_MODES, MAX_MODES, seed=23, W=1.2, H=0.9)
    small = synth.uniform_blocks(500, 40, 70, seed=24, charge=True)
    for p in (big, small):
        x, y, w, h, c = B.to_device(p, dev)
        ref = B.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, "fp32")
        got = B.grad_noalloc(x, y, w, h, c, p.W, p.H, p.Mx, p.My)
        B.sync_status(dev)
        for r, g in zip(ref, got):
            assert _close(g, r, tol)
        o = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
        for key, t in (("N", got[2]), ("gx", got[0]), ("gy", got[1])):
            r = o[key]
            assert np.max(np.abs(t.double().cpu().numpy() - r)) <= tol * np.max(np.abs(r)), key
        assert abs(float(got[3]) - o["E"]) <= tol * abs(o["E"])


def test_noalloc_rejects_sizes_beyond_its_scratch(pp):
    B = pp.binding
    dev = torch.device("cuda")
    x = torch.rand(8, device=dev)
    g = torch.empty(8, device=dev)
    L = B.lib()
    for Mx, My, n in ((257, 16, 8), (16, 300, 8)):
        prob = B.make_problem(x, x, x, x, None, 1.0, 1.0, Mx, My)
        assert L.pp_grad_noalloc(ctypes.byref(prob), 0, g.data_ptr(), g.data_ptr(), None, None,
                                 None) == 1
        assert "PP_STATIC_MAX_MODES" in L.pp_last_error().decode()
    prob = B.make_problem(x, x, x, x, None, 1.0, 1.0, 8, 8)
    prob.n = 32769
    assert L.pp_grad_noalloc(ctypes.byref(prob), 0, g.data_ptr(), g.data_ptr(), None, None, None) == 1
    assert "PP_STATIC_MAX_BLOCKS" in L.pp_last_error().decode()
    # the die range of pp_grad: a subnormal W has no finite 1/W
    for W, H in ((1e-310, 1.0), (1.0, 2e300), (float("nan"), 1.0)):
        prob = B.make_problem(x, x, x, x, None, W, H, 8, 8)
        assert L.pp_grad_noalloc(ctypes.byref(prob), 0, g.data_ptr(), g.data_ptr(), None, None,
                                 None) == 1
        assert "1e-300" in L.pp_last_error().decode()
