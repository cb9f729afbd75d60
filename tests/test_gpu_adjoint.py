"""pp_grad_adjoint (the backward pass of L = g_total E + sum_i g_block_i N_i) and
pp_coeffs_accumulate (coefficients summed over calls in FP64), through the C ABI.

The adjoint's reference is the FP64 oracle's derivative of L written out from
Sec. II-B and Eq. (aup): with w_i = g_total / 2 + g_block_i,
dL/dx_j = w_j h_j + h^b_j, h the oracle gradient of E with the placement's
coefficients a and h^b the same with the coefficients b of the charges c_i w_i;
test_gpu_autograd.py checks the same quantity against finite differences.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import series as O
from paper_2307_12041_gb300 import synth

pytestmark = pytest.mark.gpu
PRECS = ["fp32", "tf32", "bf16x3"]
# normalised max error of the adjoint: both of its terms carry the precision's error
ADJ_TOL = {"fp32": 2e-6, "tf32": 2e-3, "bf16x3": 2e-4}


def oracle_adjoint(p, g_total, g_block):
    c = np.ones(p.n) if p.c is None else p.c.astype(np.float64)
    wgt = 0.5 * g_total + (np.zeros(p.n) if g_block is None else g_block.astype(np.float64))
    a = O.coefficients(p.W, p.H, p.x, p.y, p.w, p.h, c, p.Mx, p.My)
    N, hx, hy = O.energy_grad(p.W, p.H, p.x, p.y, p.w, p.h, c, a)
    b = O.coefficients(p.W, p.H, p.x, p.y, p.w, p.h, c * wgt, p.Mx, p.My)
    _, bx, by = O.energy_grad(p.W, p.H, p.x, p.y, p.w, p.h, c, b)
    return wgt * hx + bx, wgt * hy + by, N, 0.5 * float(np.sum(N))


def nerr(got, ref):
    got = got.double().cpu().numpy() if hasattr(got, "cpu") else np.asarray(got)
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("prec", PRECS)
def test_vector_adjoint_matches_oracle(pp, prec):
    B = pp.binding
    p = synth.cell_mix(3000, 96, 80, seed=41)
    p.c = np.random.default_rng(1).uniform(0.5, 1.5, p.n).astype(np.float32)
    gb = np.random.default_rng(2).normal(size=p.n).astype(np.float32)
    gt = 0.7
    rx, ry, rN, rE = oracle_adjoint(p, gt, gb)
    dev = torch.device("cuda")
    x, y, w, h, c = B.to_device(p, dev)
    mov = np.ones(p.n, bool)
    mov[::7] = False
    gx, gy, eb, et = B.grad_adjoint(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec,
                                    g_total=torch.tensor([gt], dtype=torch.float64, device=dev),
                                    g_block=torch.from_numpy(gb).to(dev),
                                    movable=torch.from_numpy(mov).to(dev), want_energy=True)
    B.sync_status(dev)
    rx[~mov] = 0.0
    ry[~mov] = 0.0
    gxn, gyn = gx.double().cpu().numpy(), gy.double().cpu().numpy()
    assert np.all(gxn[~mov] == 0.0) and np.all(gyn[~mov] == 0.0)
    scale = max(np.max(np.abs(rx)), np.max(np.abs(ry)))
    err = max(np.max(np.abs(gxn - rx)), np.max(np.abs(gyn - ry))) / scale
    assert err <= ADJ_TOL[prec], (prec, err)
    assert nerr(eb, rN) <= B.TOLERANCE[prec]
    assert abs(float(et) - rE) <= B.TOLERANCE[prec] * abs(rE)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("sample", ["rect", "center"])
def test_scalar_adjoint_is_scaled_masked_gradient(pp, prec, sample):
    """g_block = NULL: one evaluation whose gradient is g_total * (pp_grad's), masked."""
    B = pp.binding
    p = synth.uniform_blocks(2500, 64, 72, seed=42, charge=True)
    dev = torch.device("cuda")
    x, y, w, h, c = B.to_device(p, dev)
    mov = torch.from_numpy(np.arange(p.n) % 5 != 0).to(dev)
    g = torch.tensor([-1.75], dtype=torch.float64, device=dev)
    gx, gy, eb, et = B.grad_adjoint(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec, sample, g_total=g,
                                    movable=mov, want_energy=True)
    rgx, rgy, reb, ret = B.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec, sample)
    B.sync_status(dev)
    m = mov.float()
    assert torch.equal(gx, (rgx * -1.75) * m) and torch.equal(gy, (rgy * -1.75) * m)
    # E is an FP64 atomic sum: its last bits depend on the order of the additions
    assert torch.equal(eb, reb) and abs(float(et) - float(ret)) <= 1e-12 * abs(float(ret))


def test_adjoint_rejects_bad_arguments(pp):
    B = pp.binding
    dev = torch.device("cuda")
    t = torch.rand(16, device=dev)
    g = torch.empty(16, device=dev)
    prob = B.make_problem(t, t, t, t, None, 1.0, 1.0, 8, 8)
    ws = B.workspace(prob, "fp32", dev)
    L = B.lib()
    call = lambda sample, gt, gb: L.pp_grad_adjoint(ctypes.byref(prob), 0, sample, gt, gb, None, g.data_ptr(),
                                                   g.data_ptr(), None, None, ws.data_ptr(), ws.numel(), None)
    assert call(0, None, None) == 1 and "both NULL" in L.pp_last_error().decode()
    assert call(1, None, t.data_ptr()) == 1 and "PP_RECT" in L.pp_last_error().decode()
    gt_host = torch.ones(1, dtype=torch.float64)
    assert call(0, gt_host.data_ptr(), None) == 1


@pytest.mark.parametrize("prec", PRECS)
def test_coefficients_accumulate_over_chunks_in_fp64(pp, prec):
    """a64 after adding three chunks equals the oracle's a of the whole placement,
    a_out is the rounded running sum, and a call with no blocks only rounds."""
    B = pp.binding
    p = synth.cell_mix(9000, 130, 96, seed=43)
    ref = O.coefficients(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    dev = torch.device("cuda")
    x, y, w, h, c = B.to_device(p, dev)
    a64 = torch.zeros((p.Mx, p.My), dtype=torch.float64, device=dev)
    a32 = torch.full((p.Mx, p.My), float("nan"), dtype=torch.float32, device=dev)
    cuts = [0, 2500, 2501, 9000]
    for k, (s, e) in enumerate(zip(cuts[:-1], cuts[1:])):
        B.coeffs_accumulate(x[s:e], y[s:e], w[s:e], h[s:e], None, p.W, p.H, p.Mx, p.My, a64, prec,
                            a_out=a32 if k == 2 else None)
    B.sync_status(dev)
    assert nerr(a64, ref) <= B.TOLERANCE[prec]
    assert torch.equal(a32, a64.float())
    whole = B.coeffs(x, y, w, h, None, p.W, p.H, p.Mx, p.My, prec)
    assert float((whole.double() - a64).abs().max()) <= B.TOLERANCE[prec] * float(a64.abs().max())
    a64.mul_(0.5)
    e = torch.empty(0, dtype=torch.float32, device=dev)
    B.coeffs_accumulate(e, e, e, e, None, p.W, p.H, p.Mx, p.My, a64, prec, a_out=a32)
    torch.cuda.synchronize()
    assert torch.equal(a32, a64.float())
