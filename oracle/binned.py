"""FP64 CPU oracle of the paper's binned fast scheme (arXiv 2307.12041, Sec. III-D).

TEST INFRASTRUCTURE ONLY: only the tests may import this module; it shares no code
with the CUDA library.

Steps, in the paper's order and notation (m x m uniform bins b_lj of size
w_b = W/m, h_b = H/m, centres x_l = (l + 1/2) w_b, y_j = (j + 1/2) h_b):

1. Bin density P_lj = (total area of blocks in b_lj) / (area of b_lj).  The paper
   weights a block's area by a local-smoothness rule it does not state; the
   reading taken is the literal definition: the exact overlap area of block i's
   rectangle with the bin, times its charge c_i.
2. Coefficients, Eq. (disa-a)..(disa-d), u < Mx, p < My (K = M - 1 <= m - 1):
     a'_up = sum_lj P_lj cos(u (l + 1/2) pi / m) cos(p (j + 1/2) pi / m),
     a_0p = 4 H^2 / (p^3 pi^3 m) sin(p pi / 2m) a'_0p,
     a_u0 = 4 W^2 / (u^3 pi^3 m) sin(u pi / 2m) a'_u0,
     a_up = 16 W^2 H^2 / (u p (u^2 H^2 + p^2 W^2) pi^4) sin(u pi / 2m) sin(p pi / 2m) a'_up,
     a_00 = 0  (the parenthesis of Eq. disa-c is read as cos(u (l + 1/2) pi / m)).
   The double sums are matrix products with the cosine matrices (a library primitive).
3. Bin-centre potential and field, Eq. (dis-psi1) and (dis-ksi):
     psi(l, j) = sum_up a_up cos(u (l + 1/2) pi / m) cos(p (j + 1/2) pi / m),
     xi_x(l, j) = sum_up (u pi / W) a_up sin(u (l + 1/2) pi / m) cos(p (j + 1/2) pi / m),
     xi_y(l, j) = sum_up (p pi / H) a_up cos(u (l + 1/2) pi / m) sin(p (j + 1/2) pi / m).
4. Per block, "weighting the corresponding values of its surrounding bins": the
   reading taken is bilinear interpolation between the four bin centres around the
   block centre (coordinates clamped to the outermost centres, m >= 2).  With the
   centre reading of Sec. III-C, N_i = q_i psi_i (q_i = c_i w_i h_i), the gradient of
   E = 1/2 sum_i N_i is -q_i xi_i (Sec. IV: grad N = -q xi).
"""
from __future__ import annotations

import math

import numpy as np

PI = math.pi


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def bin_density(W, H, x, y, w, h, c, m):
    """P (m x m, index [l, j]) of step 1."""
    x, y, w, h = map(_f64, (x, y, w, h))
    c = np.ones(len(x)) if c is None else _f64(c)
    wb, hb = W / m, H / m
    P = np.zeros((m, m))
    edges_x = np.arange(m + 1) * wb
    edges_y = np.arange(m + 1) * hb
    for i in range(len(x)):
        x0, x1 = x[i] - w[i] / 2, x[i] + w[i] / 2
        y0, y1 = y[i] - h[i] / 2, y[i] + h[i] / 2
        ox = np.clip(np.minimum(edges_x[1:], x1) - np.maximum(edges_x[:-1], x0), 0.0, None)
        oy = np.clip(np.minimum(edges_y[1:], y1) - np.maximum(edges_y[:-1], y0), 0.0, None)
        lx, ly = np.nonzero(ox)[0], np.nonzero(oy)[0]
        if len(lx) and len(ly):
            P[np.ix_(lx, ly)] += c[i] * np.outer(ox[lx], oy[ly])
    return P / (wb * hb)


def cos_matrix(M, m):
    """C[u, l] = cos(u (l + 1/2) pi / m), u < M."""
    return np.cos(np.outer(np.arange(M), np.arange(m) + 0.5) * PI / m)


def sin_matrix(M, m):
    return np.sin(np.outer(np.arange(M), np.arange(m) + 0.5) * PI / m)


def binned_coefficients(P, W, H, Mx, My):
    """Step 2: a (Mx x My) from the bin density P (m x m)."""
    m = P.shape[0]
    ap = cos_matrix(Mx, m) @ P @ cos_matrix(My, m).T            # a'_up
    a = np.zeros((Mx, My))
    u = np.arange(Mx, dtype=np.float64)
    p = np.arange(My, dtype=np.float64)
    su = np.sin(u * PI / (2 * m))
    sp = np.sin(p * PI / (2 * m))
    if My > 1:
        a[0, 1:] = 4 * H * H / (p[1:] ** 3 * PI ** 3 * m) * sp[1:] * ap[0, 1:]
    if Mx > 1:
        a[1:, 0] = 4 * W * W / (u[1:] ** 3 * PI ** 3 * m) * su[1:] * ap[1:, 0]
    if Mx > 1 and My > 1:
        U, Pp = u[1:, None], p[None, 1:]
        a[1:, 1:] = (16 * W * W * H * H / (U * Pp * (U * U * H * H + Pp * Pp * W * W) * PI ** 4)
                     * su[1:, None] * sp[None, 1:] * ap[1:, 1:])
    a[0, 0] = 0.0
    return a


def bin_fields(a, W, H, m):
    """Step 3: psi, xi_x, xi_y on the m x m bin centres (index [l, j])."""
    Mx, My = a.shape
    Cx, Sx = cos_matrix(Mx, m), sin_matrix(Mx, m)
    Cy, Sy = cos_matrix(My, m), sin_matrix(My, m)
    ku = np.arange(Mx) * PI / W
    lp = np.arange(My) * PI / H
    psi = Cx.T @ a @ Cy
    xi_x = Sx.T @ (ku[:, None] * a) @ Cy
    xi_y = Cx.T @ (a * lp[None, :]) @ Sy
    return psi, xi_x, xi_y


def bilinear(V, W, H, x, y):
    """Step 4: V (m x m, bin centres) at points (x, y)."""
    m = V.shape[0]
    fx = np.clip(_f64(x) / (W / m) - 0.5, 0.0, m - 1.0)
    fy = np.clip(_f64(y) / (H / m) - 0.5, 0.0, m - 1.0)
    l0 = np.minimum(np.floor(fx).astype(int), m - 2)
    j0 = np.minimum(np.floor(fy).astype(int), m - 2)
    tx, ty = fx - l0, fy - j0
    return ((1 - tx) * (1 - ty) * V[l0, j0] + tx * (1 - ty) * V[l0 + 1, j0]
            + (1 - tx) * ty * V[l0, j0 + 1] + tx * ty * V[l0 + 1, j0 + 1])


def evaluate(W, H, x, y, w, h, c, Mx, My, m):
    """The whole scheme: dict(P, a, psi, xi_x, xi_y, N, gx, gy, E)."""
    P = bin_density(W, H, x, y, w, h, c, m)
    a = binned_coefficients(P, W, H, Mx, My)
    psi, xi_x, xi_y = bin_fields(a, W, H, m)
    cc = np.ones(len(x)) if c is None else _f64(c)
    q = cc * _f64(w) * _f64(h)
    N = q * bilinear(psi, W, H, x, y)
    gx = -q * bilinear(xi_x, W, H, x, y)
    gy = -q * bilinear(xi_y, W, H, x, y)
    return dict(P=P, a=a, psi=psi, xi_x=xi_x, xi_y=xi_y, N=N, gx=gx, gy=gy, E=0.5 * float(N.sum()))
