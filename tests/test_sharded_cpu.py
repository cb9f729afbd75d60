"""The sharded evaluation (paper_2307_12041_gb300/sharded.py) as two gloo
processes on the CPU: the block partition, the one FP64 all-reduce of the
coefficient sums and the row ownership.  The library's arithmetic is replaced by
stand-ins built from the FP64 oracle (no GPU here), so what is checked is the
host logic: every block is counted once, the reduced coefficients equal the whole
placement's, each rank's gradient rows are its own blocks', and E is the whole
placement's on every rank."""
import math
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _placement():
    from paper_2307_12041_gb300 import synth
    return synth.uniform_blocks(1001, 24, 20, seed=91, W=1.2, H=0.8, charge=True)


def _textbook_G(W, H, Mx, My):
    eu = np.where(np.arange(Mx) == 0, 1.0, 2.0)
    ev = np.where(np.arange(My) == 0, 1.0, 2.0)
    k2 = (np.arange(Mx)[:, None] * math.pi / W) ** 2 + (np.arange(My)[None, :] * math.pi / H) ** 2
    k2[0, 0] = 1.0
    G = eu[:, None] * ev[None, :] / (W * H * k2)
    G[0, 0] = 0.0
    return G


class OracleOps:
    """Stand-ins for the library calls, from the FP64 oracle, on CPU tensors."""
    seen = []

    @staticmethod
    def zeros64(Mx, My, device):
        return torch.zeros((Mx, My), dtype=torch.float64, device=device)

    @staticmethod
    def accumulate(x, y, w, h, c, W, H, Mx, My, a64, prec):
        from oracle import series as O
        OracleOps.seen.append(x.numel())
        if x.numel():
            a64 += torch.from_numpy(O.coefficients(W, H, x.numpy(), y.numpy(), w.numpy(), h.numpy(),
                                                   None if c is None else c.numpy(), Mx, My))

    @staticmethod
    def round(a64, W, H, prec):
        OracleOps.a64 = a64.clone()
        return a64.float()

    @staticmethod
    def grad(x, y, w, h, c, W, H, Mx, My, prec, a):
        from oracle import series as O
        N, gx, gy = O.energy_grad(W, H, x.numpy(), y.numpy(), w.numpy(), h.numpy(),
                                  None if c is None else c.numpy(), a.double().numpy())
        return torch.from_numpy(gx), torch.from_numpy(gy), torch.from_numpy(N)

    @staticmethod
    def energy(a, W, H):
        a = a.double().numpy()
        G = _textbook_G(W, H, *a.shape)
        S = np.where(G > 0, a / np.where(G > 0, G, 1.0), 0.0)
        return torch.tensor([0.5 * float(np.sum(a * S))], dtype=torch.float64)


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    from paper_2307_12041_gb300 import sharded
    from test_sharded_cpu import OracleOps, _placement
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    p = _placement()
    s, e = sharded.block_range(p.n, world, rank)
    own = sharded.shard(p, world, rank)
    t = lambda v: torch.from_numpy(v)
    gx, gy, N, E, a = sharded.evaluate(t(own.x), t(own.y), t(own.w), t(own.h), t(own.c), p.W, p.H,
                                       p.Mx, p.My, "fp32", ops=OracleOps)
    out.put((rank, s, e, OracleOps.seen, OracleOps.a64.numpy(), gx.numpy(), gy.numpy(), N.numpy(),
             float(E)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_one_placement():
    from oracle import series as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda r: r[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = _placement()
    ref = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    # the partition: contiguous, disjoint, every block once, one accumulate per rank
    assert [(r[1], r[2]) for r in res] == [(0, 501), (501, 1001)]
    assert [r[3] for r in res] == [[501], [500]]
    for rank, s, e, _, a64, gx, gy, N, E in res:
        # the all-reduced FP64 sums are the whole placement's coefficients on every rank
        assert np.max(np.abs(a64 - ref["a"])) <= 1e-13 * np.max(np.abs(ref["a"]))
        # each rank's rows are its own blocks' (against the whole placement's a)
        for k, got in (("gx", gx), ("gy", gy), ("N", N)):
            r = ref[k][s:e]
            assert got.shape == r.shape
            assert np.max(np.abs(got - r)) <= 1e-6 * np.max(np.abs(ref[k])), (rank, k)
        assert abs(E - ref["E"]) <= 1e-6 * abs(ref["E"])
    # both ranks hold the same sums: one exchange, no per-rank drift
    assert np.array_equal(res[0][4], res[1][4])


def test_single_process_needs_no_collective():
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle import series as O
    from paper_2307_12041_gb300 import sharded
    p = _placement()
    OracleOps.seen = []
    t = lambda v: torch.from_numpy(v)
    gx, gy, N, E, a = sharded.evaluate(t(p.x), t(p.y), t(p.w), t(p.h), t(p.c), p.W, p.H, p.Mx, p.My,
                                       "fp32", ops=OracleOps)
    ref = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    assert OracleOps.seen == [p.n]
    assert np.max(np.abs(gx.numpy() - ref["gx"])) <= 1e-6 * np.max(np.abs(ref["gx"]))
    assert abs(float(E) - ref["E"]) <= 1e-6 * abs(ref["E"])


@pytest.mark.parametrize("n,world", [(10, 3), (7, 7), (5, 8), (200_000, 8), (0, 2)])
def test_block_ranges_cover_every_block_once(n, world):
    from paper_2307_12041_gb300 import sharded
    rs = [sharded.block_range(n, world, r) for r in range(world)]
    assert rs[0][0] == 0 and rs[-1][1] == n
    assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
    sizes = [e - s for s, e in rs]
    assert max(sizes) - min(sizes) <= 1
