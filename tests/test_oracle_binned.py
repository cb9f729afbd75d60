"""Pins of the binned-scheme oracle (oracle/binned.py, Sec. III-D) against the exact
series oracle and against closed forms:

* the bin density is the set of bins as charged rectangles, so its binned
  coefficients (Eq. disa) equal the exact coefficients (Eq. aup/au0/a0p) of those
  rectangles, for any placement;
* for blocks aligned to the bins, the binned coefficients equal the blocks' exact
  coefficients (the identity the paper derives Eq. disa from);
* the bin density conserves charge-weighted area;
* bin-centre psi and xi (Eq. dis-psi1, dis-ksi) equal the exact potential and field
  (Eq. psi, ksi) of the same coefficients at the bin centres;
* bilinear weighting reproduces bilinear functions exactly and is clamped at the
  die edge;
* with more bins, the scheme's per-block energies approach the exact series in the
  centre reading.
"""
import numpy as np

from oracle import binned as B
from oracle import series as O
from paper_2307_12041_gb300 import synth


def test_binned_coefficients_equal_exact_of_bin_rectangles():
    p = synth.uniform_blocks(120, 20, 18, seed=3, W=1.3, H=0.9, charge=True)
    m = 32
    P = B.bin_density(p.W, p.H, p.x, p.y, p.w, p.h, p.c, m)
    a_bin = B.binned_coefficients(P, p.W, p.H, 20, 18)
    wb, hb = p.W / m, p.H / m
    L, J = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    xs, ys = ((L + 0.5) * wb).ravel(), ((J + 0.5) * hb).ravel()
    a_ex = O.coefficients(p.W, p.H, xs, ys, np.full(m * m, wb), np.full(m * m, hb), P.ravel(), 20, 18)
    assert np.max(np.abs(a_bin - a_ex)) <= 1e-12 * np.max(np.abs(a_ex))


def test_grid_aligned_blocks_binned_equals_exact():
    m, W, H = 16, 2.0, 1.0
    g = np.random.default_rng(4)
    l0, j0 = g.integers(0, m - 3, 25), g.integers(0, m - 3, 25)
    nl, nj = g.integers(1, 4, 25), g.integers(1, 4, 25)
    w, h = nl * W / m, nj * H / m
    x, y = l0 * W / m + w / 2, j0 * H / m + h / 2
    c = g.uniform(0.5, 2.0, 25)
    P = B.bin_density(W, H, x, y, w, h, c, m)
    a_bin = B.binned_coefficients(P, W, H, 24, 24)         # modes past m - 1 included
    a_ex = O.coefficients(W, H, x, y, w, h, c, 24, 24)
    assert np.max(np.abs(a_bin[:m, :m] - a_ex[:m, :m])) <= 1e-12 * np.max(np.abs(a_ex))


def test_bin_density_conserves_area():
    p = synth.uniform_blocks(300, 8, 8, seed=9, charge=True)
    m = 40
    P = B.bin_density(p.W, p.H, p.x, p.y, p.w, p.h, p.c, m)
    area = np.sum(p.c.astype(np.float64) * p.w.astype(np.float64) * p.h.astype(np.float64))
    assert abs(P.sum() * (p.W / m) * (p.H / m) - area) < 1e-14


def test_bin_fields_equal_exact_field_at_bin_centres():
    p = synth.uniform_blocks(200, 24, 20, seed=11, W=1.2, H=0.8)
    m = 28
    a = O.coefficients(p.W, p.H, p.x, p.y, p.w, p.h, p.c, 24, 20)
    psi, xi_x, xi_y = B.bin_fields(a, p.W, p.H, m)
    L, J = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    xs, ys = ((L + 0.5) * p.W / m).ravel(), ((J + 0.5) * p.H / m).ravel()
    ps = O.potential(a, p.W, p.H, xs, ys).reshape(m, m)
    fx, fy = (v.reshape(m, m) for v in O.field(a, p.W, p.H, xs, ys))
    for got, ref in ((psi, ps), (xi_x, fx), (xi_y, fy)):
        assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_bilinear_exact_on_bilinear_functions_and_clamped():
    m, W, H = 10, 2.0, 3.0
    L, J = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    xc, yc = (L + 0.5) * W / m, (J + 0.5) * H / m
    f = lambda x, y: 1.5 - 0.7 * x + 0.3 * y + 0.25 * x * y
    V = f(xc, yc)
    g = np.random.default_rng(1)
    x = g.uniform(W / (2 * m), W - W / (2 * m), 50)
    y = g.uniform(H / (2 * m), H - H / (2 * m), 50)
    assert np.max(np.abs(B.bilinear(V, W, H, x, y) - f(x, y))) < 1e-12
    # outside the outermost centres the value is the edge's
    assert abs(B.bilinear(V, W, H, [0.0], [0.0])[0] - V[0, 0]) < 1e-15
    assert abs(B.bilinear(V, W, H, [W], [H])[0] - V[-1, -1]) < 1e-15


def test_binned_approaches_exact_centre_energies():
    p = synth.uniform_blocks(150, 16, 16, seed=21, mean_size=0.01)
    ref = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, 16, 16, sample="center")
    errs = []
    for m in (32, 64, 128, 256):
        r = B.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, 16, 16, m)
        errs.append(np.max(np.abs(r["N"] - ref["N"])) / np.max(np.abs(ref["N"])))
    assert errs[-1] < 0.05 and all(b < a for a, b in zip(errs, errs[1:])), errs
