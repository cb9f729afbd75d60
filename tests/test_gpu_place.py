"""The placement loop's kernels (Sec. IV) through the C ABI against the FP64
oracle (oracle/place.py): log-sum-exp wirelength and its gradient, the overflow
ratio, the preconditioned combination, the step norms and the Nesterov step; then
the whole loop on a scaled-down synthetic netlist, checked against the oracle's
wirelength and density gradients at the GPU's own positions at checkpoints."""
import math

import numpy as np
import pytest
import torch

from oracle import binned as OB
from oracle import place as OP
from oracle import series as OS
from paper_2307_12041_gb300 import place, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_netlist():
    n = 20_000
    p = synth.placement_cells(n, 128, 11, start_sigma=0.2)
    ptr, pins = synth.netlist(n, 12)
    return p, ptr, pins


@pytest.mark.parametrize("gamma", [0.02, 1e-3])
def test_wirelength_matches_oracle(pp, small_netlist, gamma):
    p, ptr, pins = small_netlist
    nl = pp.binding.DeviceNetlist(p.n, ptr, pins)
    x, y = torch.from_numpy(p.x).cuda(), torch.from_numpy(p.y).cuda()
    gx, gy, out = pp.binding.wirelength(nl, x, y, gamma)
    W, hp, rgx, rgy = OP.lse_wirelength(p.x, p.y, ptr, pins, gamma)
    o = out.cpu().numpy()
    assert abs(o[0] - W) <= 2e-6 * W, (o[0], W)
    assert abs(o[1] - hp) <= 1e-6 * hp, (o[1], hp)
    g = np.concatenate([gx.double().cpu().numpy(), gy.double().cpu().numpy()])
    r = np.concatenate([rgx, rgy])
    assert np.abs(g - r).max() <= 2e-5 * np.abs(r).max(), np.abs(g - r).max()


@pytest.mark.parametrize("gamma", [0.02, 1e-3])
def test_wirelength_with_long_nets_matches_oracle(pp, gamma):
    """Nets of 9 to 3,000 pins (taken by a whole warp, a pin per lane, beyond 32 pins in
    several rounds) next to short ones, against the FP64 oracle."""
    n = 6000
    p = synth.placement_cells(n, 64, 21, start_sigma=0.2)
    ptr, pins = synth.netlist(n, 22)
    g = np.random.default_rng(23)
    big = [g.choice(n, d, replace=False) for d in (9, 31, 32, 33, 64, 65, 300, 3000)]
    pins = np.concatenate([pins] + big)
    ptr = np.concatenate([ptr, ptr[-1] + np.cumsum([len(b) for b in big])])
    nl = pp.binding.DeviceNetlist(p.n, ptr, pins)
    x, y = torch.from_numpy(p.x).cuda(), torch.from_numpy(p.y).cuda()
    gx, gy, out = pp.binding.wirelength(nl, x, y, gamma)
    W, hp, rgx, rgy = OP.lse_wirelength(p.x, p.y, ptr, pins, gamma)
    o = out.cpu().numpy()
    assert abs(o[0] - W) <= 2e-6 * W, (o[0], W)
    assert abs(o[1] - hp) <= 1e-6 * hp, (o[1], hp)
    gg = np.concatenate([gx.double().cpu().numpy(), gy.double().cpu().numpy()])
    r = np.concatenate([rgx, rgy])
    assert np.abs(gg - r).max() <= 2e-5 * np.abs(r).max(), np.abs(gg - r).max()


def test_wirelength_edge_cases(pp):
    # one-pin and empty nets add nothing; a two-pin net gives +-tanh(d / 2 gamma)
    ptr = np.array([0, 1, 1, 3])
    pins = np.array([0, 1, 2])
    nl = pp.binding.DeviceNetlist(3, ptr, pins)
    x = torch.tensor([0.5, 0.2, 0.6], device="cuda")
    y = torch.tensor([0.5, 0.3, 0.3], device="cuda")
    gamma = 0.05
    gx, gy, out = pp.binding.wirelength(nl, x, y, gamma)
    d = 0.4
    t = math.tanh(d / (2 * gamma))
    assert abs(float(gx[0])) == 0.0 and abs(float(gx[2]) - t) <= 1e-6 and abs(float(gx[1]) + t) <= 1e-6
    assert abs(float(gy[1])) <= 1e-7 and abs(float(gy[2])) <= 1e-7
    W = d + 2 * gamma * math.log1p(math.exp(-d / gamma)) + 2 * gamma * math.log(2.0)
    o = out.cpu().numpy()
    assert abs(o[0] - W) <= 1e-6 and abs(o[1] - d) <= 1e-6


def test_overflow_matches_oracle(pp):
    g = np.random.default_rng(21)
    n, m = 3000, 64
    w = np.where(g.random(n) < 0.05, g.uniform(0.02, 0.08, n), g.uniform(0.001, 0.01, n)).astype(np.float32)
    h = np.where(g.random(n) < 0.05, g.uniform(0.02, 0.08, n), np.full(n, 0.004)).astype(np.float32)
    x = (w / 2 + g.random(n) * (1 - w)).astype(np.float32)
    y = (0.5 + g.normal(0, 0.1, n)).clip(h / 2, 1 - h / 2).astype(np.float32)
    t = lambda a: torch.from_numpy(a).cuda()
    for target in (1.0, 0.7):
        out, bins = pp.binding.overflow(t(x), t(y), t(w), t(h), 1.0, 1.0, m, target)
        tau = float(out.item()) * (1.0 / m) ** 2 / float(np.sum(w.astype(np.float64) * h))
        ref, D = OP.overflow(x, y, w, h, None, 1.0, 1.0, m, target)
        assert abs(tau - ref) <= 2e-5 * max(ref, 1e-3), (target, tau, ref)
        assert np.abs(bins.double().cpu().numpy() * (1.0 / m) ** 2 - D).max() <= 1e-5 * D.max()


def test_combine_norms_and_nesterov_match_oracle(pp):
    g = np.random.default_rng(5)
    n = 50_000
    f32 = lambda a: torch.from_numpy(np.asarray(a, np.float32)).cuda()
    gwx, gwy, gnx, gny = (g.normal(size=n) for _ in range(4))
    q = g.uniform(1e-6, 5e-6, n)
    deg = g.integers(0, 6, n)
    cell_ptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int32)
    mov = (g.random(n) < 0.95).astype(np.uint8)
    lam = 3.0e5
    gx, gy = pp.binding.place_combine(f32(gwx), f32(gwy), f32(gnx), f32(gny),
                                      torch.from_numpy(cell_ptr).cuda(), f32(q),
                                      torch.from_numpy(mov).cuda(), lam)
    pre = np.maximum(1.0, deg + lam * q)
    rx = np.where(mov > 0, (gwx + lam * gnx) / pre, 0.0)
    assert np.abs(gx.double().cpu().numpy() - rx).max() <= 1e-5 * np.abs(rx).max()
    # norms and one Nesterov step from identical inputs
    w = g.uniform(0.001, 0.01, n)
    h = np.full(n, 0.001)
    ux, vx, vpx = (g.uniform(0.1, 0.9, n) for _ in range(3))
    uy, vy, vpy = (g.uniform(0.1, 0.9, n) for _ in range(3))
    gpx, gpy = g.normal(size=n), g.normal(size=n)
    T = {k: f32(v) for k, v in dict(ux=ux, uy=uy, vx=vx, vy=vy, vpx=vpx, vpy=vpy, gpx=gpx, gpy=gpy,
                                      w=w, h=h).items()}
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    pp.binding.step_norms(T["vx"], T["vy"], T["vpx"], T["vpy"], gx, gy, T["gpx"], T["gpy"], norms)
    gxh, gyh = gx.double().cpu().numpy(), gy.double().cpu().numpy()
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)
    dv = np.sum((f(vx) - f(vpx)) ** 2 + (f(vy) - f(vpy)) ** 2)
    dg = np.sum((gxh - f(gpx)) ** 2 + (gyh - f(gpy)) ** 2)
    nrm = norms.cpu().numpy()
    assert abs(nrm[0] - dv) <= 1e-6 * dv and abs(nrm[1] - dg) <= 1e-6 * dg
    a_k = 2.7
    coef = (a_k - 1.0) / OP.nesterov_next_a(a_k)
    pp.binding.nesterov_step(1.0, 1.0, T["ux"], T["uy"], T["vx"], T["vy"], T["vpx"], T["vpy"], gx, gy,
                             T["gpx"], T["gpy"], T["w"], T["h"], torch.from_numpy(mov).cuda(), norms, 0.0, coef)
    alpha = math.sqrt(dv / dg)
    rux, rvx = OP.nesterov_step(f(ux), f(vx), gxh, f(w), 1.0, alpha, a_k, movable=mov)
    assert np.abs(T["ux"].double().cpu().numpy() - rux).max() <= 2e-6
    assert np.abs(T["vx"].double().cpu().numpy() - rvx).max() <= 2e-6
    assert np.array_equal(T["vpx"].cpu().numpy(), np.asarray(vx, np.float32))   # v saved as v_prev
    assert np.array_equal(T["gpx"].cpu().numpy(), gx.cpu().numpy())            # g saved as g_prev


def test_place_loop_spreads_and_gradients_match_oracle(pp):
    """150 iterations on 8,000 cells (70% utilisation, started in a cluster) and
    64 x 64 modes: the overflow falls, and at iterations 0 and 60 the GPU's
    wirelength and density gradients at the GPU's positions match the oracle."""
    n, M = 8000, 64
    p = synth.placement_cells(n, M, 31)
    ptr, pins = synth.netlist(n, 32)
    checks = {}

    def cb(k, rec, xe, ye, ux, uy):
        if k in (0, 60):
            checks[k] = (xe.cpu().numpy(), ye.cpu().numpy(), rec)

    r = place.place(p, ptr, pins, iters=150, prec="fp32", tau_stop=0.0, callback=cb)
    assert r.graph, r.graph_error                        # iterations after the first replay a graph
    taus = [t["tau"] for t in r.trace]
    assert taus[-1] < 0.8 * taus[0], (taus[0], taus[-1])
    assert all(np.isfinite([t["hpwl"] for t in r.trace]))
    sub = np.random.default_rng(3).choice(n, 300, replace=False)
    for k, (vx, vy, rec) in checks.items():
        # wirelength at the GPU's positions, with the gamma of that iteration
        gx, gy, out = pp.binding.wirelength(pp.binding.DeviceNetlist(n, ptr, pins), torch.from_numpy(vx).cuda(),
                                            torch.from_numpy(vy).cuda(), rec["gamma"])
        W, hp, rgx, _ = OP.lse_wirelength(vx, vy, ptr, pins, rec["gamma"])
        assert abs(rec["W_lse"] - W) <= 2e-6 * W and abs(rec["hpwl"] - hp) <= 1e-6 * hp
        assert np.abs(gx.double().cpu().numpy() - rgx).max() <= 2e-5 * np.abs(rgx).max()
        # density: energy and gradient of the exact series at the same positions
        ref = OS.evaluate(p.W, p.H, vx, vy, p.w, p.h, None, M, M, idx=sub)
        assert abs(rec["E"] - ref["E"]) <= 1e-5 * abs(ref["E"]), (k, rec["E"], ref["E"])


def test_place_loop_with_binned_density(pp):
    """The same loop with the paper's binned scheme (Sec. III-D) as the density term:
    the overflow falls, and at iteration 0 E matches the binned oracle at the GPU's
    positions."""
    n, M = 8000, 64
    p = synth.placement_cells(n, M, 41)
    ptr, pins = synth.netlist(n, 42)
    first = {}

    def cb(k, rec, xe, ye, ux, uy):
        if k == 0:
            first["x"], first["y"], first["E"] = xe.cpu().numpy(), ye.cpu().numpy(), rec["E"]

    r = place.place(p, ptr, pins, iters=150, prec="fp32", tau_stop=0.0, callback=cb, density="binned")
    assert r.graph, r.graph_error
    taus = [t["tau"] for t in r.trace]
    assert taus[-1] < 0.8 * taus[0], (taus[0], taus[-1])
    ref = OB.evaluate(p.W, p.H, first["x"], first["y"], p.w, p.h, None, M, M, M)
    assert abs(first["E"] - ref["E"]) <= 1e-4 * abs(ref["E"]), (first["E"], ref["E"])


def test_place_loop_with_fillers(pp):
    """Filler cells bring the total area to the target density; the given blocks'
    overflow still falls."""
    n, M = 8000, 64
    p = synth.placement_cells(n, M, 51)
    ptr, pins = synth.netlist(n, 52)
    r = place.place(p, ptr, pins, iters=150, prec="fp32", tau_stop=0.0, fillers=True)
    taus = [t["tau"] for t in r.trace]
    assert taus[-1] < 0.8 * taus[0], (taus[0], taus[-1])
    assert r.x.numel() == n and np.all(np.isfinite([t["hpwl"] for t in r.trace]))


def test_place_entry_points_reject_bad_arguments(pp):
    nl = pp.binding.DeviceNetlist(2, np.array([0, 2]), np.array([0, 1]))
    x = torch.zeros(2, device="cuda")
    with pytest.raises(pp.binding.PPError):
        pp.binding.wirelength(nl, x, x.clone(), 0.0)
    with pytest.raises(pp.binding.PPError):
        pp.binding.wirelength(nl, x, x.clone(), float("nan"))
    w = torch.full((2,), 0.1, device="cuda")
    with pytest.raises(pp.binding.PPError):
        pp.binding.overflow(x, x.clone(), w, w.clone(), 1.0, 1.0, 0)
    with pytest.raises(pp.binding.PPError):
        pp.binding.overflow(x, x.clone(), w, w.clone(), 1.0, 1.0, 16, target=-1.0)
    with pytest.raises(pp.binding.PPError):
        pp.binding.place_combine(x, x, x, x, None, w, None, -1.0)


STATE = ("ux", "uy", "vx", "vy", "vpx", "vpy", "gpx", "gpy")


@pytest.mark.parametrize("graph", [False, True], ids=["call", "graph"])
@pytest.mark.parametrize("density", ["exact", "binned"])
def test_fused_iteration_matches_separate_calls(pp, density, graph):
    """pp_place_iteration issues the same kernels in the same order as the separate
    entry points.  Two placers, one fused and one not, start each iteration from the
    same state (copied over, since the FP64 sums inside the kernels are summed in
    an order that varies from run to run); the iteration's records and new state
    then agree to rounding."""
    n, M = 8000, 64
    p = synth.placement_cells(n, M, 61)
    ptr, pins = synth.netlist(n, 62)
    A = place.Placer(p, ptr, pins, "fp32", density=density, fused=True, graph=graph)
    B = place.Placer(p, ptr, pins, "fp32", density=density, fused=False)
    A.step(), B.step()                                   # the first iteration: the same path in both
    for k in range(1, 7):
        for name in STATE:
            getattr(A, name).copy_(getattr(B, name))
        A.lam, A.gamma, A.a_k, A.hp_prev, A.d_ref = B.lam, B.gamma, B.a_k, B.hp_prev, B.d_ref
        ra, rb = A.step(), B.step()
        for key in ("tau", "W_lse", "hpwl", "E", "lambda", "gamma"):
            assert ra[key] == pytest.approx(rb[key], rel=1e-6, abs=1e-12), (k, key, ra[key], rb[key])
        for name in ("ux", "uy", "vx", "vy"):
            d = (getattr(A, name) - getattr(B, name)).abs().max().item()
            assert d <= 1e-6, (k, name, d)
        for name in ("vpx", "vpy"):                       # v of the evaluation, saved as is
            assert torch.equal(getattr(A, name), getattr(B, name)), (k, name)
        for name in ("gpx", "gpy"):
            a, b = getattr(A, name), getattr(B, name)
            d = (a - b).abs().max().item()
            assert d <= 1e-5 * b.abs().max().item(), (k, name, d)
    assert A._it is not None and B._it is None
    assert (A._it.graph is not None) == graph, A._it.graph_error


def test_fused_iteration_rejects_bad_arguments(pp):
    n, M = 500, 32
    p = synth.placement_cells(n, M, 71)
    ptr, pins = synth.netlist(n, 72)
    pl = place.Placer(p, ptr, pins, "fp32")
    pl.step()
    it = pl._fused()
    it(pl.lam, pl.gamma, 0.1)
    torch.cuda.synchronize()
    b, a = pp.binding, it.a
    with pytest.raises(b.PPError):                       # workspace too small
        b._check(b.lib().pp_place_iteration(b.ctypes.byref(a), it.ws.data_ptr(), it.ws.numel() - 256, None))
    for field, bad in (("density", 7), ("n_overflow", n + 1), ("n_overflow", -1), ("M", 0)):
        old = getattr(a, field)
        setattr(a, field, bad)
        try:
            assert b.lib().pp_place_workspace_size(b.ctypes.byref(a)) == 0, field
            with pytest.raises(b.PPError):
                b._check(b.lib().pp_place_iteration(b.ctypes.byref(a), it.ws.data_ptr(), it.ws.numel(), None))
        finally:
            setattr(a, field, old)
    old = a.scalars                                      # device scalars must be 16-byte aligned
    a.scalars = it.scal_dev.data_ptr() + 4
    try:
        with pytest.raises(b.PPError):
            b._check(b.lib().pp_place_iteration(b.ctypes.byref(a), it.ws.data_ptr(), it.ws.numel(), None))
    finally:
        a.scalars = old
    with pytest.raises(b.PPError):                       # gamma must be > 0
        it(pl.lam, 0.0, 0.1)
    eager = place.Placer(p, ptr, pins, "fp32", graph=False)
    eager.step()
    with pytest.raises(b.PPError):                       # the same check in the library call
        eager._fused()(eager.lam, 0.0, 0.1)
    b.sync_status()


@pytest.mark.parametrize("density", ["exact", "binned"])
def test_device_loop_updates_match_the_host_loop(pp, density):
    """pp_place_run's scalar update (record, penalty and smoothing updates, Nesterov
    sequence) is the host loop's: one device iteration at a time (max_iters = k + 1)
    from the host placer's state, compared with the host placer's own step."""
    n, M = 8000, 64
    p = synth.placement_cells(n, M, 61)
    ptr, pins = synth.netlist(n, 62)
    A = place.Placer(p, ptr, pins, "fp32", density=density)
    B = place.Placer(p, ptr, pins, "fp32", density=density, fused=False)
    A.step(), B.step()
    for k in range(1, 7):
        for name in STATE:
            getattr(A, name).copy_(getattr(B, name))
        A.lam, A.gamma, A.a_k, A.hp_prev, A.d_ref, A.tau = B.lam, B.gamma, B.a_k, B.hp_prev, B.d_ref, B.tau
        recs = A.run_device(k + 1, tau_stop=-1.0)
        rb = B.step()
        assert len(recs) == 1 and recs[0]["k"] == k == rb["k"], (k, recs)
        assert A.stop == "max_iters" and A.k == B.k == k + 1
        ra = recs[0]
        for key in ("lambda", "gamma"):                  # the values the iteration used
            assert ra[key] == rb[key], (k, key, ra[key], rb[key])
        for key in ("tau", "W_lse", "hpwl", "E"):
            assert ra[key] == pytest.approx(rb[key], rel=1e-6, abs=1e-12), (k, key, ra[key], rb[key])
        for name in ("lam", "gamma", "hp_prev", "tau"):  # the updated scalars
            assert getattr(A, name) == pytest.approx(getattr(B, name), rel=1e-5), (k, name)
        assert A.a_k == B.a_k                            # sqrt is correctly rounded on both sides
        for name in ("ux", "uy", "vx", "vy"):
            d = (getattr(A, name) - getattr(B, name)).abs().max().item()
            assert d <= 1e-6, (k, name, d)


@pytest.mark.parametrize("density", ["exact", "binned"])
def test_device_loop_runs_to_the_overflow_stop(pp, density):
    """The whole loop after the first iteration in one pp_place_run: it stops at the
    first iteration whose overflow is below tau_stop, with the trajectory of the host
    loop (iteration counts within two of each other, the same final HPWL to 2%)."""
    n, M = 8000, 64
    p = synth.placement_cells(n, M, 81)
    ptr, pins = synth.netlist(n, 82)
    rd = place.place(p, ptr, pins, iters=400, prec="fp32", tau_stop=0.12, density=density)
    rh = place.place(p, ptr, pins, iters=400, prec="fp32", tau_stop=0.12, density=density, device_loop=False)
    assert rd.device_loop and not rh.device_loop, rd.device_loop_error
    assert rd.stop == "converged"
    assert [r["k"] for r in rd.trace] == list(range(rd.iterations))
    assert rd.trace[-1]["tau"] < 0.12 <= min(r["tau"] for r in rd.trace[:-1])
    assert abs(rd.iterations - rh.iterations) <= 2, (rd.iterations, rh.iterations)
    assert rd.trace[-1]["hpwl"] == pytest.approx(rh.trace[-1]["hpwl"], rel=2e-2)
    for a, b in zip(rd.trace[:5], rh.trace[:5]):         # the start of the trajectory agrees closely
        assert a["hpwl"] == pytest.approx(b["hpwl"], rel=1e-4), (a, b)
    # the iteration cap: exactly `iters` records, the last one k = iters - 1
    rc = place.place(p, ptr, pins, iters=9, prec="fp32", tau_stop=0.0, density=density)
    assert rc.device_loop and rc.stop == "max_iters" and rc.iterations == 9
    assert [r["k"] for r in rc.trace] == list(range(9))


def test_device_loop_stop_codes_and_rejections(pp):
    n, M = 2000, 32
    p = synth.placement_cells(n, M, 91)
    ptr, pins = synth.netlist(n, 92)
    b = pp.binding
    pl = place.Placer(p, ptr, pins, "fp32", density="binned")
    pl.step()
    it = pl._fused()

    def run(**kw):
        st = b.PlaceState(lam=pl.lam, gamma=pl.gamma, a_k=pl.a_k, hpwl_prev=pl.hp_prev, d_ref=pl.d_ref,
                          tau=pl.tau, k=pl.k, stop=0, run_count=0)
        sc = b.PlaceSchedule(max_iters=50, reserved=0, tau_stop=0.0, bin_area=pl.bin_area, area_mov=pl.area_mov,
                             bin_w=pl.bin_w)
        for key, v in kw.items():
            setattr(st if hasattr(st, key) else sc, key, v)
        return it.run(st, sc)

    ux = pl.ux.clone()
    for bad_state, code in ((dict(k=0), 5), (dict(d_ref=0.0), 5), (dict(lam=float("nan")), 3),
                            (dict(gamma=1e-60), 3), (dict(stop=1), 1), (dict(k=50), 2)):
        out, recs = run(**bad_state)                     # refused on the device: no iteration runs
        assert out.stop == code and out.run_count == 0 and recs == [], (bad_state, out.stop)
    assert torch.equal(pl.ux, ux)
    for bad in (dict(max_iters=0), dict(max_iters=(1 << 24) + 1), dict(bin_area=0.0), dict(area_mov=-1.0),
                dict(bin_w=float("inf")), dict(tau_stop=float("nan"))):
        with pytest.raises(b.PPError):                   # refused on the host
            run(**bad)
    st = b.PlaceState(lam=pl.lam, gamma=pl.gamma, a_k=pl.a_k, hpwl_prev=pl.hp_prev, d_ref=pl.d_ref, tau=pl.tau,
                      k=pl.k)
    sc = b.PlaceSchedule(max_iters=5, tau_stop=0.0, bin_area=pl.bin_area, area_mov=pl.area_mov, bin_w=pl.bin_w)
    trace = torch.zeros((5, 64), dtype=torch.uint8, device="cuda")
    sdev = torch.zeros(96, dtype=torch.uint8, device="cuda")
    L = b.lib()
    with pytest.raises(b.PPError):                       # state must be 16-byte aligned device memory
        b._check(L.pp_place_run(b.ctypes.byref(it.a), b.ctypes.byref(sc), sdev.data_ptr() + 8, trace.data_ptr(),
                                it.ws.data_ptr(), it.ws.numel(), None))
    with pytest.raises(b.PPError):                       # host memory
        b._check(L.pp_place_run(b.ctypes.byref(it.a), b.ctypes.byref(sc), b.ctypes.addressof(st), trace.data_ptr(),
                                it.ws.data_ptr(), it.ws.numel(), None))
    with pytest.raises(b.PPError):                       # trace NULL
        b._check(L.pp_place_run(b.ctypes.byref(it.a), b.ctypes.byref(sc), sdev.data_ptr(), None,
                                it.ws.data_ptr(), it.ws.numel(), None))
    with pytest.raises(b.PPError):                       # workspace too small
        b._check(L.pp_place_run(b.ctypes.byref(it.a), b.ctypes.byref(sc), sdev.data_ptr(), trace.data_ptr(),
                                it.ws.data_ptr(), it.ws.numel() - 256, None))
    torch.cuda.synchronize()
    b.sync_status()


def test_device_loop_stops_on_the_device_status_word(pp):
    """A bounded wait that ran out (the library's failure-path probe) leaves the status
    word set; the device loop makes the iteration in flight, then stops with
    device_error instead of carrying on, and pp_sync_status reports the timeout."""
    n, M = 2000, 32
    p = synth.placement_cells(n, M, 93)
    ptr, pins = synth.netlist(n, 94)
    pp.binding.sync_status()
    pl = place.Placer(p, ptr, pins, "fp32", density="binned")
    pl.step()
    pp.binding.check_wait_timeout(1_000_000)
    recs = pl.run_device(100, tau_stop=0.0)
    assert pl.stop == "device_error" and len(recs) == 1 and recs[0]["k"] == 1, (pl.stop, len(recs))
    with pytest.raises(pp.binding.PPError) as err:
        pp.binding.sync_status()
    assert err.value.status == 4
    recs = pl.run_device(5, tau_stop=0.0)                # cleared: the loop runs on
    assert pl.stop == "max_iters" and [r["k"] for r in recs] == [2, 3, 4]
