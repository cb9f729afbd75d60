"""The binned fast scheme on the GPU (pp_binned_grad) against its FP64 oracle
(oracle/binned.py): coefficients, per-block energies, gradients and E, for
uniform and clustered placements, W != H, charges, and modes up to m."""
import numpy as np
import pytest
import torch

from oracle import binned as B
from paper_2307_12041_gb300 import synth

pytestmark = pytest.mark.gpu

# density by FP32 atomics, FP32 transforms (FFTs for m a power of two, direct sums
# otherwise) in both precisions
BINNED_TOL = {"fp32": 2e-5, "tf32": 2e-5}

CASES = [
    # n, Mx, My, m, W, H, charge, kind
    (600, 40, 48, 64, 1.0, 1.0, False, "uniform"),
    (500, 64, 64, 64, 1.3, 0.8, True, "uniform"),
    (3000, 100, 90, 128, 1.0, 1.0, False, "mix"),
    (1, 2, 2, 2, 1.0, 1.0, False, "uniform"),
    (20000, 256, 200, 512, 1.0, 1.0, False, "mix"),          # warp FFT, R = 16
    (30000, 300, 260, 1024, 1.1, 0.9, True, "mix"),           # warp FFT, R = 32
    (2000, 100, 120, 256, 1.0, 1.0, False, "mix"),            # block FFT, 8 radix-2 stages
    (700, 50, 60, 96, 1.2, 0.9, True, "uniform"),             # m not a power of two: direct sums
    (5, 3, 3, 3, 1.0, 1.0, False, "uniform"),
    (4000, 90, 100, 100, 1.0, 1.0, False, "mix"),
]


def nerr(got, ref):
    scale = np.max(np.abs(ref))
    return float(np.max(np.abs(np.asarray(got, np.float64) - ref)) / scale) if scale > 0 else 0.0


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}_m{c[3]}")
@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_binned_matches_oracle(pp, case, prec):
    n, Mx, My, m, W, H, charge, kind = case
    if kind == "uniform":
        p = synth.uniform_blocks(n, Mx, My, seed=n + m, W=W, H=H, charge=charge, mean_size=0.01)
    else:
        p = synth.cell_mix(n, Mx, My, seed=n + m, W=W, H=H)
    ref = B.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, Mx, My, m)
    x, y, w, h, c = pp.binding.to_device(p, torch.device("cuda"))
    gx, gy, N, E, a = pp.binding.binned_grad(x, y, w, h, c, p.W, p.H, Mx, My, m, prec)
    pp.binding.sync_status()
    tol = BINNED_TOL[prec]
    assert nerr(a.cpu().numpy(), ref["a"]) <= tol
    assert nerr(N.cpu().numpy(), ref["N"]) <= tol
    g = np.concatenate([gx.cpu().numpy(), gy.cpu().numpy()])
    assert nerr(g, np.concatenate([ref["gx"], ref["gy"]])) <= tol
    assert abs(float(E.item()) - ref["E"]) <= tol * abs(ref["E"])


@pytest.mark.parametrize("m", [512, 1024, 256, 100])
def test_binned_out_of_die_blocks_match_oracle(pp, m):
    """Blocks overhanging the die, wider than it, or outside it (only the part inside
    the die is binned, in the oracle as on the GPU): large blocks take the difference
    array with their column range clamped to the grid; m = 512, 1024 add its prefix
    sums in the first row transform, 256 in the separate kernel, 100 uses direct sums."""
    p = synth.out_of_die_blocks(3000, 64, 48, seed=40 + m, W=1.2, H=0.9)
    ref = B.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, 64, 48, m)
    x, y, w, h, c = pp.binding.to_device(p, torch.device("cuda"))
    gx, gy, N, E, a = pp.binding.binned_grad(x, y, w, h, c, p.W, p.H, 64, 48, m, "fp32")
    pp.binding.sync_status()
    tol = BINNED_TOL["fp32"]
    assert nerr(a.cpu().numpy(), ref["a"]) <= tol
    assert nerr(N.cpu().numpy(), ref["N"]) <= tol
    g = np.concatenate([gx.cpu().numpy(), gy.cpu().numpy()])
    assert nerr(g, np.concatenate([ref["gx"], ref["gy"]])) <= tol
    assert abs(float(E.item()) - ref["E"]) <= tol * abs(ref["E"])


@pytest.mark.parametrize("m", [512, 100])
def test_binned_density_is_deterministic(pp, m):
    """The bin density is summed in 64-bit fixed point, so the order in which the
    atomics land does not matter: two runs give the same coefficients, per-block
    energies and gradients bit for bit (E, a sum over CTAs in FP64, to rounding)."""
    p = synth.out_of_die_blocks(3000, 64, 48, seed=40 + m, W=1.2, H=0.9)
    x, y, w, h, c = pp.binding.to_device(p, torch.device("cuda"))
    r1 = pp.binding.binned_grad(x, y, w, h, c, p.W, p.H, 64, 48, m, "fp32")
    r2 = pp.binding.binned_grad(x, y, w, h, c, p.W, p.H, 64, 48, m, "fp32")
    for name, a, b in zip(("gx", "gy", "N", "E", "a"), r1, r2):
        if name == "E":
            assert float(a.item()) == pytest.approx(float(b.item()), rel=1e-13)
        else:
            assert torch.equal(a, b), name


def test_binned_rejects_bad_bins(pp):
    p = synth.uniform_blocks(10, 8, 8, seed=1)
    x, y, w, h, c = pp.binding.to_device(p, torch.device("cuda"))
    with pytest.raises(pp.binding.PPError):
        pp.binding.binned_grad(x, y, w, h, c, p.W, p.H, 8, 8, 4)       # m < Mx
    with pytest.raises(pp.binding.PPError):
        pp.binding.binned_grad(x, y, w, h, c, p.W, p.H, 8, 8, 16, "bf16x3")
