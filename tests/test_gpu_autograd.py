"""The autograd wrapper (energy forward, adjoint gradient backward with the
coefficients recomputed) against pp_grad, and against finite differences of the
FP64 energy on sampled coordinates.

Finite differences.  E = 1/2 sum_{u,p} G_up S_up^2 with S = sum_i c_i X_i Y_i^T
(rectangle integrals, textbook weights G = e_u e_p / (W H (k_u^2 + l_p^2))).
Moving block j by d along x changes S by D = c_j (X_j(x_j + d) - X_j(x_j)) Y_j^T,
so E(x_j + d) - E = sum G (S D + D^2 / 2) exactly; the central difference
[dE(+d) - dE(-d)] / (2d) at d = 1e-6 is evaluated in FP64 from the oracle's S
for each sampled coordinate, without re-evaluating the whole placement.
"""
import math

import numpy as np
import pytest
import torch

from oracle import series as O
from paper_2307_12041_gb300 import synth

pytestmark = pytest.mark.gpu
PI = math.pi


def textbook_G(W, H, Mx, My):
    eu = np.where(np.arange(Mx) == 0, 1.0, 2.0)
    ep = np.where(np.arange(My) == 0, 1.0, 2.0)
    k2 = (np.arange(Mx)[:, None] * PI / W) ** 2 + (np.arange(My)[None, :] * PI / H) ** 2
    k2[0, 0] = 1.0
    G = eu[:, None] * ep[None, :] / (W * H * k2)
    G[0, 0] = 0.0
    return G


def fd_gradients(p, coords, d=1e-6):
    """Central differences of the FP64 energy for (block, axis) pairs."""
    a = O.coefficients(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    G = textbook_G(p.W, p.H, p.Mx, p.My)
    with np.errstate(divide="ignore", invalid="ignore"):
        S = np.where(G > 0, a / np.where(G > 0, G, 1.0), 0.0)
    c = np.ones(p.n) if p.c is None else p.c.astype(np.float64)
    px, py, pw, ph = (np.asarray(v, dtype=np.float64) for v in (p.x, p.y, p.w, p.h))
    out = []
    for j, axis in coords:
        # positions widened to float64 before the displacement d is added
        if axis == 0:
            X0, _ = O.rect_integrals([px[j]], [pw[j]], p.W, p.Mx)
            Xp, _ = O.rect_integrals([px[j] + d], [pw[j]], p.W, p.Mx)
            Xm, _ = O.rect_integrals([px[j] - d], [pw[j]], p.W, p.Mx)
            Y, _ = O.rect_integrals([py[j]], [ph[j]], p.H, p.My)
            Dp = c[j] * np.outer(Xp[0] - X0[0], Y[0])
            Dm = c[j] * np.outer(Xm[0] - X0[0], Y[0])
        else:
            X, _ = O.rect_integrals([px[j]], [pw[j]], p.W, p.Mx)
            Y0, _ = O.rect_integrals([py[j]], [ph[j]], p.H, p.My)
            Yp, _ = O.rect_integrals([py[j] + d], [ph[j]], p.H, p.My)
            Ym, _ = O.rect_integrals([py[j] - d], [ph[j]], p.H, p.My)
            Dp = c[j] * np.outer(X[0], Yp[0] - Y0[0])
            Dm = c[j] * np.outer(X[0], Ym[0] - Y0[0])
        dEp = np.sum(G * (S * Dp + 0.5 * Dp * Dp))
        dEm = np.sum(G * (S * Dm + 0.5 * Dm * Dm))
        out.append((dEp - dEm) / (2 * d))
    return np.array(out)


def run_autograd(pp, p, prec, movable=None):
    dev = torch.device("cuda")
    x, y, w, h, c = pp.binding.to_device(p, dev)
    x = x.clone().requires_grad_(True)
    y = y.clone().requires_grad_(True)
    mov = None if movable is None else torch.from_numpy(movable).to(dev)
    E = pp.binding.PoissonEnergy.apply(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec, "rect", mov)
    (2.0 * E).backward()          # grad_out = 2 scales the adjoint
    return float(E.item()), x.grad.detach(), y.grad.detach()


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3"])
def test_autograd_equals_grad_entry_point(pp, prec):
    p = synth.uniform_blocks(3000, 80, 72, seed=31, charge=True)
    E, gx, gy = run_autograd(pp, p, prec)
    dev = torch.device("cuda")
    x, y, w, h, c = pp.binding.to_device(p, dev)
    rgx, rgy, _, rE = pp.binding.grad(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec)
    tol = pp.binding.TOLERANCE[prec]
    assert abs(E - float(rE)) <= tol * abs(float(rE))
    scale = float(torch.maximum(rgx.abs().max(), rgy.abs().max()))
    assert float((gx - 2 * rgx).abs().max()) <= 2 * tol * scale
    assert float((gy - 2 * rgy).abs().max()) <= 2 * tol * scale


def test_fixed_blocks_get_no_gradient(pp):
    p = synth.workload(3, n=20000)          # cells + 500 fixed macros
    p.Mx = p.My = 128
    _, gx, gy = run_autograd(pp, p, "tf32", movable=p.movable)
    fixed = torch.from_numpy(~p.movable).cuda()
    assert float(gx[fixed].abs().max()) == 0.0 and float(gy[fixed].abs().max()) == 0.0
    assert float(gx[~fixed].abs().max()) > 0.0


@pytest.fixture(scope="module")
def cells_fixed_macros():
    """2,000,000 cells + 500 fixed macros, 1024 x 1024 modes; 1,000 seeded
    (block, axis) samples among the movable cells and their FD gradients."""
    p = synth.workload(3)
    g = np.random.default_rng(2307)
    blocks = g.choice(np.flatnonzero(p.movable), 1000, replace=False)
    axes = g.integers(0, 2, 1000)
    coords = list(zip(blocks.tolist(), axes.tolist()))
    return p, coords, fd_gradients(p, coords)


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "tf32"])
def test_autograd_finite_differences_full_size(pp, cells_fixed_macros, prec):
    p, coords, fd = cells_fixed_macros
    _, gx, gy = run_autograd(pp, p, prec, movable=p.movable)
    gxh = gx.double().cpu().numpy() / 2
    gyh = gy.double().cpu().numpy() / 2
    got = np.array([gxh[j] if ax == 0 else gyh[j] for j, ax in coords])
    err = np.max(np.abs(got - fd)) / np.max(np.abs(fd))
    assert err <= pp.binding.TOLERANCE[prec], (prec, err)


def oracle_L(p, gw, x, y):
    """L = sum_i g_i N_i (rectangle reading) in FP64 at positions (x, y)."""
    a = O.coefficients(p.W, p.H, x, y, p.w, p.h, p.c, p.Mx, p.My)
    N = O.energy_grad(p.W, p.H, x, y, p.w, p.h, p.c, a)[0]
    return float(np.dot(gw, N))


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3"])
def test_block_energies_adjoint_matches_fd(pp, prec):
    """Vector-output adjoint: d(sum_i g_i N_i)/d(x, y) for a random g against central
    differences of the FP64 oracle's sum_i g_i N_i on 30 sampled coordinates."""
    p = synth.uniform_blocks(400, 40, 48, seed=77, charge=True)
    gw = np.random.default_rng(3).normal(size=p.n)
    dev = torch.device("cuda")
    x, y, w, h, c = pp.binding.to_device(p, dev)
    x = x.clone().requires_grad_(True)
    y = y.clone().requires_grad_(True)
    N = pp.binding.PoissonBlockEnergies.apply(x, y, w, h, c, p.W, p.H, p.Mx, p.My, prec)
    (N * torch.from_numpy(gw).to(dev, torch.float32)).sum().backward()
    gx, gy = x.grad.double().cpu().numpy(), y.grad.double().cpu().numpy()
    g = np.random.default_rng(4)
    coords = list(zip(g.choice(p.n, 30, replace=False).tolist(), g.integers(0, 2, 30).tolist()))
    px, py = p.x.astype(np.float64), p.y.astype(np.float64)
    d = 1e-6
    fd, got = [], []
    for j, ax in coords:
        xp, yp, xm, ym = px.copy(), py.copy(), px.copy(), py.copy()
        if ax == 0:
            xp[j] += d
            xm[j] -= d
        else:
            yp[j] += d
            ym[j] -= d
        fd.append((oracle_L(p, gw, xp, yp) - oracle_L(p, gw, xm, ym)) / (2 * d))
        got.append(gx[j] if ax == 0 else gy[j])
    fd, got = np.array(fd), np.array(got)
    err = np.max(np.abs(got - fd)) / np.max(np.abs(fd))
    assert err <= 2 * pp.binding.TOLERANCE[prec] + 1e-6, (prec, err)


def test_block_energies_scalar_case_is_energy_gradient(pp):
    """g = 1/2 for every block: d(1/2 sum N_i)/dx = dE/dx, the gradient pp_grad returns."""
    p = synth.uniform_blocks(1000, 64, 48, seed=8)
    dev = torch.device("cuda")
    x, y, w, h, c = pp.binding.to_device(p, dev)
    x = x.clone().requires_grad_(True)
    y = y.clone().requires_grad_(True)
    N = pp.binding.PoissonBlockEnergies.apply(x, y, w, h, c, p.W, p.H, p.Mx, p.My, "fp32")
    (0.5 * N).sum().backward()
    rgx, rgy, _, _ = pp.binding.grad(x.detach(), y.detach(), w, h, c, p.W, p.H, p.Mx, p.My, "fp32")
    scale = float(torch.maximum(rgx.abs().max(), rgy.abs().max()))
    assert float((x.grad - rgx).abs().max()) <= 2e-6 * scale
    assert float((y.grad - rgy).abs().max()) <= 2e-6 * scale
