"""The sharded evaluation (one placement's blocks shared out over ranks, sharded.py)
on the GPU with the library's own operations.  One GPU runs the ranks one after
another, with no rank waiting on another: each rank's FP64 coefficient sum is added
into one array, which is what the all-reduce sums over processes.  Then every
rank's rows are evaluated against the rounded coefficients.  The concatenated rows,
the coefficients and E are compared with the FP64 oracle on the whole placement."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import series as O  # noqa: E402
from paper_2307_12041_gb300 import binding, sharded, synth  # noqa: E402

from test_gpu_parity import check  # noqa: E402


@pytest.mark.parametrize("prec,world", [("fp32", 3), ("tf32", 3), ("bf16x3", 2), ("tf32", 1)])
def test_ranks_in_turn_match_the_oracle(prec, world):
    p = synth.cell_mix(6000, 96, 80, seed=71 + world, W=1.1, H=0.9)
    dev = torch.device("cuda")
    ops = sharded.LibraryOps
    a64 = ops.zeros64(p.Mx, p.My, dev)
    parts = [binding.to_device(sharded.shard(p, world, r), dev) for r in range(world)]
    for x, y, w, h, c in parts:                 # the all-reduce's sum, rank by rank
        ops.accumulate(x, y, w, h, c, p.W, p.H, p.Mx, p.My, a64, prec)
    a = ops.round(a64, p.W, p.H, prec)
    rows = [ops.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec, a) for x, y, w, h, c in parts]
    E = ops.energy(a, p.W, p.H)
    binding.sync_status()
    out = {"a": a, "N": torch.cat([r[2] for r in rows]), "gx": torch.cat([r[0] for r in rows]),
           "gy": torch.cat([r[1] for r in rows]), "E": float(E.item())}
    ref = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    # the flat bound (FP32, BF16x3) and, for the tensor-core precisions, every element
    # within its forward-error bound, as in test_gpu_parity
    check(out, ref, binding.TOLERANCE[prec], label=f"{prec} x{world}", p=p, prec=prec)


def test_single_process_evaluate_is_the_sum_of_its_parts():
    """sharded.evaluate in one process (no torch.distributed) equals the ranks run in
    turn with world = 1: the same library calls."""
    p = synth.cell_mix(3000, 64, 64, seed=9)
    dev = torch.device("cuda")
    x, y, w, h, c = binding.to_device(p, dev)
    gx, gy, eb, E, a = sharded.evaluate(x, y, w, h, c, p.W, p.H, p.Mx, p.My, "tf32")
    ref = binding.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, "tf32", a=a)
    assert torch.equal(gx, ref[0]) and torch.equal(gy, ref[1]) and torch.equal(eb, ref[2])
    assert abs(float(E.item()) - float(binding.energy_from_coeffs(a, p.W, p.H).item())) <= 1e-12 * abs(float(E.item()))
