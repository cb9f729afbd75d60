"""FP64 CPU oracle of the analytical Poisson series (arXiv 2307.12041, Sec. III).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  The product path (the CUDA library
and its Python binding) never calls it and shares no code with it.

What it computes, in the paper's notation (die R = [0, W] x [0, H], blocks with
centres (x_i, y_i), sizes (w_i, h_i), charge density c_i, default 1):

* Eq. (global density) and Eq. (rho): rho = sum_i c_i theta_i(x) theta_i(y) minus
  its mean.  The charge c_i generalises the paper's unit density (theta = 1); the
  mean only feeds the (0, 0) mode, which Eq. (a-a) sets to zero.
* Eq. (aup), (au0), (a0p): the coefficients a_{u,p} as the literal sums of
  differences of sines, with a_{0,0} = 0 (Eq. a-a).
* Eq. (psi) and Eq. (ksi): potential and field, truncated to u < Mx, p < My
  (Sec. III-B: "take the first K terms").
* Per-block energy.  Sec. II-B defines N(v) = 1/2 sum_i N_i with N_i the energy of
  charge i.  Rectangle reading (default): N_i = c_i * integral over block i of psi,
  the energy of the exact block density, so that E = 1/2 integral of rho psi.
  Centre reading: N_i = q_i psi(x_i, y_i) with q_i = c_i w_i h_i (Sec. III-C
  substitutes the centre).
* Gradient.  Sec. IV: grad N = -q xi.  Rectangle reading: dE/dx_i =
  -c_i * integral over block i of xi_x (the field of Eq. ksi integrated over the
  block), which is exactly the derivative of E; centre reading: -q_i xi(x_i, y_i).

Every step is a plain numpy float64 expression; the contraction over blocks is a
matrix product (a library primitive) accumulated chunk by chunk over blocks
only to bound memory.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

PI = math.pi
_CHUNK = 4096


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def _threads() -> int:
    return max(1, int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1)))


# ---------------------------------------------------------------------------
# One-dimensional pieces
# ---------------------------------------------------------------------------

def sine_differences(centre, size, L, M):
    """D[i, u] = sin(u pi (x_i + w_i/2) / L) - sin(u pi (x_i - w_i/2) / L), u = 0..M-1.

    The bracketed factors of Eq. (aup), (au0) and (a0p), evaluated literally
    (column u = 0 is identically zero)."""
    centre = _f64(centre)[:, None]
    size = _f64(size)[:, None]
    k = np.arange(M, dtype=np.float64)[None, :] * PI / L
    return np.sin(k * (centre + 0.5 * size)) - np.sin(k * (centre - 0.5 * size))


def cosine_differences(centre, size, L, M):
    """C[i, u] = cos(u pi (x_i - w_i/2) / L) - cos(u pi (x_i + w_i/2) / L)."""
    centre = _f64(centre)[:, None]
    size = _f64(size)[:, None]
    k = np.arange(M, dtype=np.float64)[None, :] * PI / L
    return np.cos(k * (centre - 0.5 * size)) - np.cos(k * (centre + 0.5 * size))


def rect_integrals(centre, size, L, M):
    """(Ic, Is): Ic[i, u] = int theta_i(t) cos(u pi t / L) dt and
    Is[i, u] = int theta_i(t) sin(u pi t / L) dt over the block's extent.

    Antiderivatives of cos and sin: Ic = D * L / (u pi) (u >= 1), Ic[:, 0] = size;
    Is = C * L / (u pi) (u >= 1), Is[:, 0] = 0."""
    D = sine_differences(centre, size, L, M)
    C = cosine_differences(centre, size, L, M)
    scale = np.zeros(M)
    scale[1:] = L / (np.arange(1, M) * PI)
    Ic = D * scale[None, :]
    Is = C * scale[None, :]
    Ic[:, 0] = _f64(size)
    Is[:, 0] = 0.0
    return Ic, Is


# ---------------------------------------------------------------------------
# Coefficients a_{u,p}: Eq. (a-a), (aup), (au0), (a0p)
# ---------------------------------------------------------------------------

def _charges(p_c, n):
    return np.ones(n) if p_c is None else _f64(p_c)


def _chunks(n, size=_CHUNK):
    return [(s, min(n, s + size)) for s in range(0, n, size)]


def coefficients(W, H, x, y, w, h, c, Mx, My):
    """Truncated coefficient matrix a (Mx x My), float64.

    a[u, p] for u, p >= 1 (Eq. aup):
        4 W^2 H^2 / ((u^2 H^2 + p^2 W^2) u p pi^4) * sum_i c_i Dx[i,u] Dy[i,p]
    a[u, 0], u >= 1 (Eq. au0):  2 W^2 / (u^3 pi^3 H) * sum_i c_i h_i Dx[i,u]
    a[0, p], p >= 1 (Eq. a0p):  2 H^2 / (p^3 pi^3 W) * sum_i c_i w_i Dy[i,p]
    a[0, 0] = 0 (Eq. a-a).
    """
    W = float(W)
    H = float(H)
    n = len(x)
    cc = _charges(c, n)
    x, y, w, h = map(_f64, (x, y, w, h))

    def part(se):
        s, e = se
        Dx = sine_differences(x[s:e], w[s:e], W, Mx)
        Dy = sine_differences(y[s:e], h[s:e], H, My)
        cD = cc[s:e, None] * Dx
        S = cD.T @ Dy                       # sum_i c_i Dx[i,u] Dy[i,p]
        ax = (cc[s:e] * h[s:e]) @ Dx        # sum_i c_i h_i Dx[i,u]
        ay = (cc[s:e] * w[s:e]) @ Dy        # sum_i c_i w_i Dy[i,p]
        return S, ax, ay

    S = np.zeros((Mx, My))
    ax = np.zeros(Mx)
    ay = np.zeros(My)
    with ThreadPoolExecutor(_threads()) as ex:
        for Sp, axp, ayp in ex.map(part, _chunks(n)):
            S += Sp
            ax += axp
            ay += ayp

    a = np.zeros((Mx, My))
    u = np.arange(Mx, dtype=np.float64)
    p = np.arange(My, dtype=np.float64)
    if Mx > 1 and My > 1:
        U = u[1:, None]
        P = p[None, 1:]
        pref = 4.0 * W * W * H * H / ((U * U * H * H + P * P * W * W) * U * P * PI ** 4)
        a[1:, 1:] = pref * S[1:, 1:]
    if Mx > 1:
        a[1:, 0] = 2.0 * W * W / (u[1:] ** 3 * PI ** 3 * H) * ax[1:]
    if My > 1:
        a[0, 1:] = 2.0 * H * H / (p[1:] ** 3 * PI ** 3 * W) * ay[1:]
    a[0, 0] = 0.0
    return a


# ---------------------------------------------------------------------------
# Potential and field at points: Eq. (psi), Eq. (ksi)
# ---------------------------------------------------------------------------

def potential(a, W, H, px, py):
    """psi(px, py) = sum_{u,p} a[u,p] cos(u pi x / W) cos(p pi y / H)  (Eq. psi)."""
    Mx, My = a.shape
    cx = np.cos(np.outer(_f64(px), np.arange(Mx)) * PI / W)
    cy = np.cos(np.outer(_f64(py), np.arange(My)) * PI / H)
    return np.einsum("iu,up,ip->i", cx, a, cy)


def field(a, W, H, px, py):
    """(xi_x, xi_y) at points (Eq. ksi):
    xi_x = sum (u pi / W) a sin(u pi x / W) cos(p pi y / H),
    xi_y = sum (p pi / H) a cos(u pi x / W) sin(p pi y / H)."""
    Mx, My = a.shape
    ku = np.arange(Mx) * PI / W
    lp = np.arange(My) * PI / H
    ax = np.outer(_f64(px), ku)
    ay = np.outer(_f64(py), lp)
    xi_x = np.einsum("iu,up,ip->i", np.sin(ax) * ku[None, :], a, np.cos(ay))
    xi_y = np.einsum("iu,up,ip->i", np.cos(ax), a, np.sin(ay) * lp[None, :])
    return xi_x, xi_y


# ---------------------------------------------------------------------------
# Per-block energy and gradient
# ---------------------------------------------------------------------------

def energy_grad(W, H, x, y, w, h, c, a, sample="rect", idx=None):
    """Per-block energy N_i and gradient (dE/dx_i, dE/dy_i) for the blocks `idx`
    (default all), given the coefficient matrix `a` of the whole placement.

    sample="rect": N_i = c_i Ix_i^T a Iy_i (the block integral of psi);
                   dE/dx_i = -c_i sum (u pi/W) a Jx_i,u Iy_i,p (block integral of xi_x),
                   dE/dy_i = -c_i sum (p pi/H) a Ix_i,u Jy_i,p.
    sample="center": N_i = q_i psi(x_i, y_i), gradient = -q_i xi(x_i, y_i),
                   q_i = c_i w_i h_i.
    Returns (N, gx, gy) as float64 arrays over `idx`.
    """
    W = float(W)
    H = float(H)
    n = len(x)
    idx = np.arange(n) if idx is None else np.asarray(idx)
    cc = _charges(c, n)[idx]
    xs, ys, ws, hs = (_f64(v)[idx] for v in (x, y, w, h))
    Mx, My = a.shape
    ku = np.arange(Mx) * PI / W
    lp = np.arange(My) * PI / H
    m = len(idx)
    N = np.zeros(m)
    gx = np.zeros(m)
    gy = np.zeros(m)

    def part(se):
        s, e = se
        if sample == "rect":
            Ix, Jx = rect_integrals(xs[s:e], ws[s:e], W, Mx)
            Iy, Jy = rect_integrals(ys[s:e], hs[s:e], H, My)
            T = Ix @ a
            n_ = cc[s:e] * np.sum(T * Iy, axis=1)
            gx_ = -cc[s:e] * np.sum(((Jx * ku[None, :]) @ a) * Iy, axis=1)
            gy_ = -cc[s:e] * np.sum(T * (Jy * lp[None, :]), axis=1)
        elif sample == "center":
            q = cc[s:e] * ws[s:e] * hs[s:e]
            psi = potential(a, W, H, xs[s:e], ys[s:e])
            xi_x, xi_y = field(a, W, H, xs[s:e], ys[s:e])
            n_, gx_, gy_ = q * psi, -q * xi_x, -q * xi_y
        else:
            raise ValueError(sample)
        return s, e, n_, gx_, gy_

    with ThreadPoolExecutor(_threads()) as ex:
        for s, e, n_, gx_, gy_ in ex.map(part, _chunks(m, 2048)):
            N[s:e] = n_
            gx[s:e] = gx_
            gy[s:e] = gy_
    return N, gx, gy


def evaluate(W, H, x, y, w, h, c, Mx, My, sample="rect", idx=None):
    """Coefficients, per-block energy, total energy E = 1/2 sum_i N_i (Sec. II-B)
    and gradient.  E sums all blocks; N, gx, gy are returned for `idx`."""
    a = coefficients(W, H, x, y, w, h, c, Mx, My)
    N, gx, gy = energy_grad(W, H, x, y, w, h, c, a, sample, idx)
    if idx is None:
        E = 0.5 * float(np.sum(N))
    else:
        E = 0.5 * float(np.sum(energy_grad(W, H, x, y, w, h, c, a, sample)[0]))
    return dict(a=a, N=N, gx=gx, gy=gy, E=E)


def total_energy(W, H, x, y, w, h, c, Mx, My, sample="rect"):
    """E = 1/2 sum_i N_i for the whole placement."""
    a = coefficients(W, H, x, y, w, h, c, Mx, My)
    N = energy_grad(W, H, x, y, w, h, c, a, sample)[0]
    return 0.5 * float(np.sum(N))
