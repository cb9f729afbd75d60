"""Pins of the placement-loop oracle (oracle/place.py) against facts that hold
independently of its code: the log-sum-exp bounds around the half-perimeter
wirelength, the two-pin closed form, the gamma -> 0 limit, central finite
differences of the FP64 wirelength, translation invariance of every net, overflow
values of placements worked out by hand, and the Nesterov sequence's first terms."""
import math

import numpy as np
import pytest

from oracle import place as P


def random_netlist(n, r, seed, dmax=6):
    g = np.random.default_rng(seed)
    deg = g.integers(2, dmax + 1, r)
    ptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)
    pins = np.concatenate([g.choice(n, d, replace=False) for d in deg]).astype(np.int64)
    x, y = g.uniform(0, 1, n), g.uniform(0, 1, n)
    return x, y, ptr, pins, deg


def brute_hpwl(x, y, ptr, pins):
    return sum(np.ptp(x[pins[a:b]]) + np.ptp(y[pins[a:b]]) for a, b in zip(ptr[:-1], ptr[1:]))


@pytest.mark.parametrize("gamma", [0.3, 0.01, 1e-4])
def test_lse_brackets_hpwl(gamma):
    x, y, ptr, pins, deg = random_netlist(200, 150, 1)
    W, hp, _, _ = P.lse_wirelength(x, y, ptr, pins, gamma)
    ref = brute_hpwl(x, y, ptr, pins)
    assert abs(hp - ref) <= 1e-12 * ref
    # each log-sum lies between the max and the max + gamma ln |e|: 4 of them per net
    assert ref - 1e-12 <= W <= ref + 4 * gamma * np.log(deg).sum() + 1e-12


def test_lse_two_pin_closed_form():
    gamma = 0.05
    x = np.array([0.31, 0.74])
    y = np.array([0.5, 0.5])
    W, _, gx, gy = P.lse_wirelength(x, y, [0, 2], [0, 1], gamma)
    d = abs(x[1] - x[0])
    # gamma ln(e^{a/g} + e^{b/g}) = max + gamma ln(1 + e^{-|a-b|/g}), same for -x
    expect = d + 2 * gamma * math.log1p(math.exp(-d / gamma)) + 2 * gamma * math.log(2.0)
    assert abs(W - expect) <= 1e-14
    # d/dx1 of |x1 - x0| smoothed: tanh(d / (2 gamma)) for the right pin
    assert abs(gx[1] - math.tanh(d / (2 * gamma))) <= 1e-14 and abs(gx[0] + gx[1]) <= 1e-15
    assert np.all(gy == 0.0)


def test_lse_gradient_finite_differences():
    x, y, ptr, pins, _ = random_netlist(60, 40, 2)
    gamma, d = 0.07, 1e-6
    _, _, gx, gy = P.lse_wirelength(x, y, ptr, pins, gamma)
    for i in range(0, 60, 7):
        for coord, g in ((x, gx), (y, gy)):
            c0 = coord[i]
            coord[i] = c0 + d
            wp = P.lse_wirelength(x, y, ptr, pins, gamma)[0]
            coord[i] = c0 - d
            wm = P.lse_wirelength(x, y, ptr, pins, gamma)[0]
            coord[i] = c0
            assert abs((wp - wm) / (2 * d) - g[i]) <= 1e-7


def test_lse_translation_invariance():
    x, y, ptr, pins, _ = random_netlist(300, 400, 3)
    W0, _, gx, gy = P.lse_wirelength(x, y, ptr, pins, 0.02)
    W1 = P.lse_wirelength(x + 0.123, y - 0.04, ptr, pins, 0.02)[0]
    assert abs(W1 - W0) <= 1e-10 * W0
    assert abs(gx.sum()) <= 1e-10 and abs(gy.sum()) <= 1e-10


def test_overflow_by_hand():
    # 4 x 4 bins on the unit die; a block exactly on bins [0, 2) x [0, 2) has density 1
    w = h = np.array([0.5])
    tau, D = P.overflow([0.25], [0.25], w, h, None, 1.0, 1.0, 4)
    assert tau == 0.0 and abs(D[:2, :2] - 1 / 16).max() < 1e-15 and D.sum() == pytest.approx(0.25)
    # two copies stacked: each of the 4 bins holds twice its area; excess = one copy
    tau, _ = P.overflow([0.25, 0.25], [0.25, 0.25], np.r_[w, w], np.r_[h, h], None, 1.0, 1.0, 4)
    assert tau == pytest.approx(0.5, abs=1e-15)
    # one copy at target density 0.5: half of its area is excess
    tau, _ = P.overflow([0.25], [0.25], w, h, None, 1.0, 1.0, 4, target=0.5)
    assert tau == pytest.approx(0.5, abs=1e-15)
    # a fixed block counts as occupancy but not as movable area
    tau, _ = P.overflow([0.25, 0.25], [0.25, 0.25], np.r_[w, w], np.r_[h, h], [True, False], 1.0, 1.0, 4)
    assert tau == pytest.approx(1.0, abs=1e-15)


def test_nesterov_sequence_and_clamp():
    a1 = P.nesterov_next_a(1.0)
    assert a1 == pytest.approx((1 + math.sqrt(5)) / 2, abs=1e-15)
    assert P.nesterov_next_a(a1) == pytest.approx((1 + math.sqrt(4 * a1 * a1 + 1)) / 2, abs=1e-15)
    u = v = np.array([0.5, 0.5, 0.02])
    g = np.array([1.0, -1.0, 1.0])
    w = np.array([0.1, 0.1, 0.02])
    un, vn = P.nesterov_step(u, v, g, w, 1.0, 0.2, 1.0)
    # first step: momentum (a0 - 1) / a1 = 0, so v1 = u1; the third block stops at w/2
    assert np.allclose(un, [0.3, 0.7, 0.01]) and np.allclose(vn, un)
    un2, vn2 = P.nesterov_step(un, vn, np.zeros(3), w, 1.0, 0.2, a1, movable=[True, True, False])
    a2 = P.nesterov_next_a(a1)
    assert np.allclose(un2[:2], un[:2]) and np.allclose(vn2[:2], un[:2])   # zero gradient: no move
    assert un2[2] == vn[2]                                                 # fixed


def test_fillers_fill_to_target_density():
    """place.with_fillers (host-side input preparation): the added cells bring the
    total area to within one filler of target * W * H, are movable and lie inside
    the die."""
    from paper_2307_12041_gb300 import place, synth
    p = synth.placement_cells(5000, 64, 3)
    q = place.with_fillers(p, 1.0, 7)
    k = q.n - p.n
    assert k > 0 and q.movable[p.n:].all()
    fa = float(q.w[-1]) * float(q.h[-1])
    total = float(np.sum(q.w.astype(np.float64) * q.h))
    assert 1.0 - fa <= total <= 1.0 + 1e-6
    assert np.all(q.x - q.w / 2 >= 0) and np.all(q.x + q.w / 2 <= 1 + 1e-6)
