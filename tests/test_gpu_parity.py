"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Error measure per output vector (coefficients a, per-block energy N, gradient
gx, gy): max |gpu - oracle| / max |oracle|, bounded by binding.TOLERANCE[prec];
the total energy E is compared relatively.  Inputs are seeded and synthetic.
"""
import math

import numpy as np
import pytest
import torch

from oracle import series as O
from paper_2307_12041_gb300 import synth
from parity_bounds import BOUND_PARAMS, bound_ratios

pytestmark = pytest.mark.gpu


def nerr(got, ref):
    got = np.asarray(got, dtype=np.float64).reshape(ref.shape)
    scale = np.max(np.abs(ref))
    return float(np.max(np.abs(got - ref)) / scale) if scale > 0 else float(np.max(np.abs(got)))


def gerr(gx, gy, ref):
    """Gradient error normalised by the gradient's scale: max over blocks and both
    components of |g - g_ref| / max over blocks and components of |g_ref|."""
    rx, ry = ref["gx"], ref["gy"]
    scale = max(np.max(np.abs(rx)), np.max(np.abs(ry)))
    d = max(np.max(np.abs(np.asarray(gx, np.float64).reshape(rx.shape) - rx)),
            np.max(np.abs(np.asarray(gy, np.float64).reshape(ry.shape) - ry)))
    return float(d / scale) if scale > 0 else float(d)


def check(out, ref, tol, keys=("a", "N", "grad"), label="", p=None, prec=None, sample="rect",
          flat=None):
    """Normalised max error of each output <= tol (the flat bound), and, for the
    tensor-core precisions when the placement `p` is given, every element within
    its forward-error bound (error_bounds).  TF32's flat bound applies only where
    `flat` is set (the workloads): without cancellation its normalised error is
    a few operand roundings, but a placement whose coefficients cancel (blocks
    wider than the die, a few hundred blocks) makes the normalised error grow with
    sum |terms| / |sum|, which only the element-wise bound follows."""
    if flat is None:
        flat = prec != "tf32"
    errs = {}
    for k in keys:
        if k == "grad":
            errs[k] = gerr(out["gx"].double().cpu().numpy(), out["gy"].double().cpu().numpy(), ref)
        else:
            errs[k] = nerr(out[k].double().cpu().numpy(), ref[k])
    errs["E"] = abs(out["E"] - ref["E"]) / max(abs(ref["E"]), 1e-300)
    if flat:
        bad = {k: v for k, v in errs.items() if not v <= tol}
        assert not bad, f"{label} errors above {tol:.1e}: {bad} (all: {errs})"
    if p is not None and prec in BOUND_PARAMS:
        ratios = bound_ratios(out, ref, p, prec, sample)
        bad = {k: v for k, v in ratios.items() if not v <= 1.0}
        assert not bad, f"{label}: error / forward-error bound above 1: {bad} (all: {ratios}, flat: {errs})"
    return errs


def placement(n, Mx, My, seed, W=1.0, H=1.0, charge=False, kind="uniform"):
    if kind == "uniform":
        return synth.uniform_blocks(n, Mx, My, seed, W, H, charge=charge)
    return synth.cell_mix(n, Mx, My, seed, W, H)


SHAPES = [
    # n, Mx, My, W, H, charge, kind
    (2000, 64, 64, 1.0, 1.0, False, "uniform"),     # the small workload
    (1, 1, 1, 1.0, 1.0, False, "uniform"),
    (1, 7, 5, 2.0, 0.5, True, "uniform"),
    (37, 5, 130, 1.0, 1.0, True, "uniform"),
    (300, 129, 33, 1.7, 0.9, True, "uniform"),
    (4099, 200, 257, 1.0, 1.0, False, "mix"),
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"n{s[0]}_{s[1]}x{s[2]}")
def test_parity_with_oracle(pp, shape):
    n, Mx, My, W, H, charge, kind = shape
    p = placement(n, Mx, My, seed=100 + n, W=W, H=H, charge=charge, kind=kind)
    ref = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, Mx, My)
    for prec in pp.binding.available_precisions():
        out = pp.binding.evaluate(p, prec=prec)
        # the first shape is the small workload: TF32's flat bound applies there too
        check(out, ref, pp.binding.TOLERANCE[prec], label=f"{prec} {shape}", p=p, prec=prec,
              flat=True if shape == SHAPES[0] else None)


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3"])
def test_center_sampling_parity(pp, prec):
    if prec not in pp.binding.available_precisions():
        pytest.skip("precision not built")
    p = placement(1500, 48, 72, seed=7, W=1.3, H=0.8, charge=True)
    ref = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My, sample="center")
    out = pp.binding.evaluate(p, prec=prec, sample="center")
    check(out, ref, pp.binding.TOLERANCE[prec], label=f"center {prec}", p=p, prec=prec, sample="center")


def test_zero_blocks(pp):
    dev = torch.device("cuda")
    e = torch.empty(0, dtype=torch.float32, device=dev)
    for prec in pp.binding.available_precisions():
        a = pp.binding.coeffs(e, e, e, e, None, 1.0, 1.0, 8, 9, prec)
        assert a.shape == (8, 9) and float(a.abs().max()) == 0.0
        gx, gy, eb, et = pp.binding.grad(e, e, e, e, None, 1.0, 1.0, 8, 9, prec)
        assert gx.numel() == 0 and float(et.item()) == 0.0


def test_given_coefficients_match_internal(pp):
    p = placement(3000, 96, 80, seed=3, charge=True)
    dev = torch.device("cuda")
    x, y, w, h, c = pp.binding.to_device(p, dev)
    for prec in pp.binding.available_precisions():
        a = pp.binding.coeffs(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec)
        g1 = pp.binding.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec)
        g2 = pp.binding.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec, a=a)
        e2 = pp.binding.energy(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec, a=a)
        tol = pp.binding.TOLERANCE[prec]
        for t1, t2 in ((g1[0], g2[0]), (g1[1], g2[1]), (g1[2], g2[2]), (g1[2], e2[0])):
            assert float((t1 - t2).abs().max()) <= tol * float(t1.abs().max())
        assert abs(float(g1[3]) - float(e2[1])) <= tol * abs(float(g1[3]))


def test_block_linearity_and_permutation(pp):
    """Coefficients are a sum over blocks: a(A u B) = a(A) + a(B) (the chunked
    accumulation a multi-GPU split would all-reduce), and block order is irrelevant."""
    p = placement(5000, 128, 128, seed=9)
    dev = torch.device("cuda")
    x, y, w, h, c = pp.binding.to_device(p, dev)
    for prec in pp.binding.available_precisions():
        tol = pp.binding.TOLERANCE[prec]
        a = pp.binding.coeffs(x, y, w, h, c, 1.0, 1.0, 128, 128, prec)
        k = 1937
        a1 = pp.binding.coeffs(x[:k], y[:k], w[:k], h[:k], None, 1.0, 1.0, 128, 128, prec)
        a2 = pp.binding.coeffs(x[k:], y[k:], w[k:], h[k:], None, 1.0, 1.0, 128, 128, prec)
        assert float((a - a1 - a2).abs().max()) <= tol * float(a.abs().max())
        perm = torch.randperm(p.n, generator=torch.Generator().manual_seed(1)).to(dev)
        ap = pp.binding.coeffs(x[perm], y[perm], w[perm], h[perm], None, 1.0, 1.0, 128, 128, prec)
        assert float((a - ap).abs().max()) <= tol * float(a.abs().max())


def test_max_mode_counts(pp):
    p = placement(64, 4096, 4096, seed=12, charge=True)
    ref = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    for prec in pp.binding.available_precisions():
        out = pp.binding.evaluate(p, prec=prec)
        check(out, ref, pp.binding.TOLERANCE[prec], label=f"4096^2 {prec}", p=p, prec=prec)


def test_invalid_pointers_are_rejected(pp):
    dev = torch.device("cuda")
    x = torch.rand(10, device=dev)
    host = torch.rand(10)
    with pytest.raises(ValueError):
        pp.binding.coeffs(x, host, x, x, None, 1.0, 1.0, 4, 4)
    ctypes = __import__("ctypes")
    prob = pp.binding.make_problem(x, x, x, x, None, 1.0, 1.0, 4, 4)
    prob.y = host.data_ptr()                     # a host address: must be refused, not launched
    a = torch.empty(16, device=dev)
    ws = pp.binding.workspace(prob, "fp32", dev)
    st = pp.binding.lib().pp_coeffs(ctypes.byref(prob), 0, a.data_ptr(), ws.data_ptr(),
                                    ws.numel(), None)
    assert st == 1
    st = pp.binding.lib().pp_coeffs(ctypes.byref(prob), 0, a.data_ptr(), ws.data_ptr(), 16, None)
    assert st in (1, 2)


# ---------------------------------------------------------------------------
# Full-size throughput workload (200k blocks, 512 x 512 modes): coefficients in
# full, energies and gradients on a seeded sample of blocks.
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def big():
    p = synth.workload(1)
    a = O.coefficients(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    idx = np.sort(np.random.default_rng(5).choice(p.n, 2000, replace=False))
    N, gx, gy = O.energy_grad(p.W, p.H, p.x, p.y, p.w, p.h, p.c, a, idx=idx)
    E = 0.5 * float(np.sum(O.energy_grad(p.W, p.H, p.x, p.y, p.w, p.h, p.c, a)[0]))
    return p, a, idx, dict(N=N, gx=gx, gy=gy, E=E)


# Bound on the relative error of the total energy: E = 1/2 sum a S is quadratic in
# the coefficients, so about twice their normalised error (FP32: the per-block
# FP64 sum; TF32, BF16x3: from the FP32 coefficients of the tensor-core contraction).
E_TOL = {"fp32": 1e-6, "tf32": 2e-4, "bf16x3": 2e-5}


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3"])
def test_full_size_workload_sampled(pp, big, prec):
    if prec not in pp.binding.available_precisions():
        pytest.skip("precision not built")
    p, a_ref, idx, ref = big
    out = pp.binding.evaluate(p, prec=prec)
    tol = pp.binding.TOLERANCE[prec]
    ea = nerr(out["a"].double().cpu().numpy(), a_ref)
    assert ea <= tol, (prec, "a", ea)
    ti = torch.from_numpy(idx).cuda()
    e = nerr(out["N"][ti].double().cpu().numpy(), ref["N"])
    assert e <= tol, (prec, "N", e)
    e = gerr(out["gx"][ti].double().cpu().numpy(), out["gy"][ti].double().cpu().numpy(), ref)
    assert e <= tol, (prec, "grad", e)
    e = abs(out["E"] - ref["E"]) / abs(ref["E"])
    assert e <= E_TOL[prec], (prec, "E", e)
    if prec == "fp32":
        # E from the GPU's per-block energies equals the GPU's FP64 total
        assert abs(out["E"] - 0.5 * float(out["N"].double().sum())) <= 1e-6 * abs(out["E"])


def test_energy_from_coefficients(pp, big):
    """pp_energy_from_coeffs on the oracle's coefficients reproduces the oracle's
    1/2 sum_i N_i (the identity 1/2 sum_i N_i = 1/2 sum_uv a_uv S_uv, S = a / G)."""
    p, a_ref, _, ref = big
    E = float(pp.binding.energy_from_coeffs(torch.from_numpy(a_ref.astype(np.float32)).cuda(), p.W, p.H).item())
    assert abs(E - ref["E"]) <= 1e-6 * abs(ref["E"])


# ---------------------------------------------------------------------------
# 1,000,000 blocks, 1024 x 1024 modes (the BF16x3 workload): coefficients in full
# and 2,000 sampled blocks' energies and gradients.
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def million():
    p = synth.workload(2)
    a = O.coefficients(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    idx = np.sort(np.random.default_rng(6).choice(p.n, 2000, replace=False))
    N, gx, gy = O.energy_grad(p.W, p.H, p.x, p.y, p.w, p.h, p.c, a, idx=idx)
    return p, a, idx, dict(N=N, gx=gx, gy=gy)


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["bf16x3", "fp32", "tf32"])
def test_million_block_workload_sampled(pp, million, prec):
    p, a_ref, idx, ref = million
    out = pp.binding.evaluate(p, prec=prec)
    tol = pp.binding.TOLERANCE[prec]
    assert nerr(out["a"].double().cpu().numpy(), a_ref) <= tol
    ti = torch.from_numpy(idx).cuda()
    assert nerr(out["N"][ti].double().cpu().numpy(), ref["N"]) <= tol
    assert gerr(out["gx"][ti].double().cpu().numpy(), out["gy"][ti].double().cpu().numpy(), ref) <= tol


def grid_aligned(n_side=24, W=1.0, H=1.0, seed=5):
    """Blocks whose centres sit on 1/16 and 1/32 fractions of the die and whose
    sizes are 1/8, 1/16, 1/32 of it: the phase steps 16 pi s, 16 pi t of the
    generators' recurrences land exactly on 0, pi/2, pi, 3 pi/2 (the boundaries
    between their two forms), next to random blocks."""
    g = np.random.default_rng(seed)
    k = np.arange(1, 32)
    xs = np.concatenate([k / 32.0, g.uniform(0.05, 0.95, n_side)]) * W
    ys = np.concatenate([k[::-1] / 32.0, g.uniform(0.05, 0.95, n_side)]) * H
    sizes = np.array([1 / 8, 1 / 16, 1 / 32, 1 / 64])
    w = sizes[np.arange(len(xs)) % 4] * W
    h = sizes[(np.arange(len(xs)) + 1) % 4] * H
    xs = np.clip(xs, w / 2, W - w / 2)
    ys = np.clip(ys, h / 2, H - h / 2)
    f32 = lambda a: np.asarray(a, np.float32)
    return synth.Placement(W=W, H=H, x=f32(xs), y=f32(ys), w=f32(w), h=f32(h), c=None,
                           Mx=300, My=280, name="grid-aligned")


def test_grid_aligned_phase_steps(pp):
    p = grid_aligned()
    ref = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    for prec in pp.binding.available_precisions():
        out = pp.binding.evaluate(p, prec=prec)
        check(out, ref, pp.binding.TOLERANCE[prec], label=f"{prec} grid-aligned", p=p, prec=prec)


def split_tile_rows(n, My, sms, rows=128, vc=256, grid_max=256):
    """Blocks of the energy kernel's row tiles that are cut between two CTAs: the
    (tile, pass) units are divided into equal ranges, one per CTA (grid = the
    smaller of the tile count, the SM count and grid_max)."""
    tiles = (n + rows - 1) // rows
    nvc = (My + vc - 1) // vc
    grid = min(tiles, sms, grid_max)
    U = tiles * nvc
    cut = set()
    for b in range(1, grid):
        ub = U * b // grid
        if ub % nvc:
            cut.add(ub // nvc)
    return sorted(cut), [t * rows + r for t in sorted(cut) for r in range(rows) if t * rows + r < n]


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_split_energy_tiles_and_determinism(pp, prec):
    """The rows of tiles cut between two CTAs of the energy kernel (their two parts
    meet through the workspace) against the FP64 oracle, and two identical calls give
    bitwise identical coefficients, per-block energies and gradients."""
    n, M = 40_000, 512                       # 313 tiles of 128 rows, two 256-column passes each
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tiles, rows = split_tile_rows(n, M, sms)
    assert len(tiles) > 10
    p = synth.cell_mix(n, M, M, 97)
    sub = np.array(rows[::7] + [rows[-1]])
    ref = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, M, M, idx=sub)
    out1 = pp.binding.evaluate(p, prec=prec)
    out2 = pp.binding.evaluate(p, prec=prec)
    tol = pp.binding.TOLERANCE[prec]
    N = out1["N"].double().cpu().numpy()[sub]
    gx = out1["gx"].double().cpu().numpy()[sub]
    gy = out1["gy"].double().cpu().numpy()[sub]
    assert nerr(N, ref["N"]) <= tol
    assert gerr(gx, gy, ref) <= tol
    for k in ("a", "N", "gx", "gy"):
        assert torch.equal(out1[k], out2[k]), k


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3"])
def test_grad_replays_from_a_cuda_graph(pp, prec):
    """pp_grad captured into a CUDA graph (fixed input, output and workspace buffers)
    and replayed after the inputs change gives the results of a direct call."""
    p = synth.cell_mix(5000, 96, 80, 17)
    q = synth.cell_mix(5000, 96, 80, 18)
    dev = torch.device("cuda")
    x, y, w, h, c = pp.binding.to_device(p, dev)
    n = p.n
    outs = (torch.empty(n, device=dev), torch.empty(n, device=dev), torch.empty(n, device=dev),
            torch.empty(1, dtype=torch.float64, device=dev))
    pp.binding.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec, out=outs)    # workspace, attributes
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            pp.binding.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec, out=outs)
    torch.cuda.synchronize()
    for src in (q, p):                   # new inputs in the captured buffers, then the old ones
        x.copy_(torch.from_numpy(src.x))
        y.copy_(torch.from_numpy(src.y))
        w.copy_(torch.from_numpy(src.w))
        h.copy_(torch.from_numpy(src.h))
        g.replay()
        torch.cuda.synchronize()
        ref = pp.binding.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec)
        for a, b in zip(outs[:3], ref[:3]):
            assert torch.equal(a, b)
        assert abs(float(outs[3]) - float(ref[3])) <= 1e-12 * abs(float(ref[3]))
    pp.binding.sync_status()


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_launch_counts_and_kernel_timing(pp, prec):
    """Every launch is counted whether or not timing is on; with timing on each
    kernel class also reports device time, and the results do not change."""
    p = synth.cell_mix(3000, 64, 64, 23)
    x, y, w, h, c = pp.binding.to_device(p, torch.device("cuda"))
    b = pp.binding
    ref = b.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec)
    b.timing_collect()
    for _ in range(3):
        b.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec)
    torch.cuda.synchronize()
    counts = b.timing_collect()
    assert {k: v[0] for k, v in counts.items()} == {"prep": 3, "coeff": 3, "finish": 3, "energy": 3}
    assert all(v[1] == 0.0 for v in counts.values())
    b.timing_enable(True)
    try:
        got = b.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec)
        torch.cuda.synchronize()
    finally:
        b.timing_enable(False)
    timed = b.timing_collect()
    assert all(v[0] == 1 and v[1] > 0.0 for v in timed.values())
    for g, r in zip(got[:3], ref[:3]):
        assert torch.equal(g, r)


# ---------------------------------------------------------------------------
# Blocks the workload generators never make: overhanging an edge, centres below
# 0 or beyond W / H, wider than the die, far outside (the literal closed forms,
# i.e. the mirror fold pinned in test_oracle_pins.py).
# ---------------------------------------------------------------------------

OUT_OF_DIE = [
    # n, Mx, My, W, H, sample
    (600, 96, 80, 1.3, 0.7, "rect"),
    (2501, 300, 257, 1.0, 1.0, "rect"),
    (777, 64, 130, 0.6, 1.9, "center"),
]


@pytest.mark.parametrize("case", OUT_OF_DIE, ids=lambda s: f"n{s[0]}_{s[1]}x{s[2]}_{s[5]}")
@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3"])
def test_out_of_die_blocks_match_oracle(pp, case, prec):
    if prec not in pp.binding.available_precisions():
        pytest.skip("precision not built")
    n, Mx, My, W, H, sample = case
    p = synth.out_of_die_blocks(n, Mx, My, seed=300 + n, W=W, H=H)
    inside = (p.x - p.w / 2 >= 0) & (p.x + p.w / 2 <= W) & (p.y - p.h / 2 >= 0) & (p.y + p.h / 2 <= H)
    assert inside.mean() < 0.2 and np.any(p.x < 0) and np.any(p.x > 2 * W) and np.any(p.w > W)
    ref = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, Mx, My, sample=sample)
    out = pp.binding.evaluate(p, prec=prec, sample=sample)
    check(out, ref, pp.binding.TOLERANCE[prec], label=f"out-of-die {prec} {case}", p=p, prec=prec,
          sample=sample)
