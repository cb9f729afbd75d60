"""pp_descent_step against its restatement in oracle/rng.py: the Philox4x32-10 /
Box-Muller normals and the clamped update, on blocks with fixed ones among them."""
import numpy as np
import pytest
import torch

from oracle import rng
from paper_2307_12041_gb300 import synth

pytestmark = pytest.mark.gpu


def test_descent_step_matches_reference(pp):
    p = synth.workload(3, n=5000)          # cells and fixed macros
    g = np.random.default_rng(4)
    gx = g.normal(0, 1e-3, p.n).astype(np.float32)
    gy = g.normal(0, 1e-3, p.n).astype(np.float32)
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    x, y, w, h = t(p.x), t(p.y), t(p.w), t(p.h)
    lr, sigma, seed, step = 3.0, 2e-3, 2307_12041 + 99, 17
    pp.binding.descent_step(x, y, w, h, t(gx), t(gy), p.W, p.H, lr, sigma, seed, step,
                            movable=t(p.movable))
    pp.binding.sync_status()
    xr, yr = rng.descent_step(p.W, p.H, p.x, p.y, p.w, p.h, gx, gy, p.movable, lr, sigma, seed, step)
    # FP32 update vs FP64 reference: the normals differ by ~1e-6 relative
    assert np.max(np.abs(x.cpu().numpy() - xr)) < 2e-6
    assert np.max(np.abs(y.cpu().numpy() - yr)) < 2e-6
    fixed = ~p.movable
    assert np.array_equal(x.cpu().numpy()[fixed], p.x[fixed])
    # the jitter itself: sigma-scaled normals recovered where no clamp applied
    moved = (x.cpu().numpy() - (p.x - lr * gx)) / sigma
    nrm = rng.descent_normals(p.n, seed, step)[0]
    inside = p.movable & (np.abs(xr - np.clip(xr, p.w / 2 + 1e-6, p.W - p.w / 2 - 1e-6)) == 0)
    assert np.max(np.abs(moved[inside] - nrm[inside])) < 5e-3      # float32 positions ~1e-7 / 2e-3


def test_descent_step_rejects_bad_arguments(pp):
    z = torch.zeros(8, dtype=torch.float32, device="cuda")
    with pytest.raises(pp.binding.PPError):
        pp.binding.descent_step(z, z, z, z, z, z, 0.0, 1.0, 1.0, 0.0, 1, 0)
    with pytest.raises(pp.binding.PPError):
        pp.binding.descent_step(z, z, z, z, z, z, 1.0, 1.0, float("nan"), 0.0, 1, 0)
