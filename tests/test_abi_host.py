"""Host-side checks of the C ABI: the library builds, loads, exports every symbol
that include/pp.h declares, sizes its workspace, and rejects bad arguments
before touching the GPU.  No kernel is launched here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2307_12041_gb300 import binding, build_lib
    build_lib.build()
    return binding.lib()


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pp_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("pp_coeffs", "pp_energy", "pp_grad", "pp_workspace_size", "pp_last_error",
                 "pp_sync_status"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_symbols():
        assert hasattr(L, name), name


def _prob(**kw):
    from paper_2307_12041_gb300.binding import Problem
    d = dict(W=1.0, H=1.0, n=10, x=None, y=None, w=None, h=None, c=None, Mx=16, My=16)
    d.update(kw)
    return Problem(d["W"], d["H"], d["n"], d["x"], d["y"], d["w"], d["h"], d["c"], d["Mx"], d["My"])


def test_workspace_size_scales_and_rejects_invalid(L):
    ws = lambda p, prec=0: L.pp_workspace_size(ctypes.byref(p), prec)
    a = ws(_prob(n=1000))
    b = ws(_prob(n=2000))
    assert a > 0 and b > a
    assert ws(_prob(n=0)) > 0
    assert ws(_prob(Mx=64, My=64)) > ws(_prob(Mx=16, My=16))
    for bad in (dict(W=0.0), dict(H=-1.0), dict(W=float("nan")), dict(W=float("inf")), dict(W=1e-310),
                dict(n=-1), dict(Mx=0), dict(My=4097), dict(n=2 ** 31)):
        assert ws(_prob(**bad)) == 0, bad
        assert L.pp_last_error().decode() != ""
    assert L.pp_workspace_size(ctypes.byref(_prob()), 7) == 0
    assert L.pp_workspace_size(None, 0) == 0


def test_calls_reject_bad_problems_before_any_launch(L):
    vp = ctypes.c_void_p
    for bad in (dict(W=0.0), dict(n=-5), dict(Mx=5000), dict(x=None, n=3)):
        p = _prob(**bad)
        assert L.pp_coeffs(ctypes.byref(p), 0, vp(16), vp(256), 1 << 20, None) == 1
        assert L.pp_energy(ctypes.byref(p), 0, 0, None, vp(16), None, vp(256), 1 << 20, None) == 1
        assert L.pp_grad(ctypes.byref(p), 0, 0, None, vp(16), vp(16), None, None, vp(256),
                         1 << 20, None) == 1
    assert L.pp_coeffs(None, 0, None, None, 0, None) == 1
    assert "NULL" in L.pp_last_error().decode()
    assert L.pp_coeffs(ctypes.byref(_prob()), 9, vp(16), vp(256), 1 << 20, None) == 1


def test_version_string(L):
    v = L.pp_version().decode()
    assert "sm_103a" in v


def test_place_workspace_size_host_only(L):
    """pp_place_workspace_size reads sizes only: it grows with the blocks and the
    modes and rejects bad densities, overflow counts and mode counts."""
    from paper_2307_12041_gb300.binding import Netlist, PlaceIterationArgs
    nl = Netlist(1000, 300, None, None, None, None)

    def size(n_cells=1000, **kw):
        nl.n_cells = n_cells
        d = dict(W=1.0, H=1.0, M=64, density=0, prec=0, n_overflow=min(1000, n_cells))
        d.update(kw)
        a = PlaceIterationArgs(ctypes.pointer(nl), d["W"], d["H"], d["M"], d["density"], d["prec"], 0,
                               d["n_overflow"])
        return L.pp_place_workspace_size(ctypes.byref(a))

    base = size()
    assert base > 0 and size(n_cells=2000) > base and size(M=128) > base
    assert size(density=1) > 0 and size(prec=1) > 0
    for bad in (dict(density=2), dict(n_overflow=1001), dict(n_overflow=-1), dict(M=0), dict(W=0.0),
                dict(density=1, M=1)):
        assert size(**bad) == 0, bad
        assert L.pp_last_error().decode() != ""
    assert L.pp_place_workspace_size(None) == 0


def test_place_run_rejects_bad_schedules_on_the_host(L):
    """pp_place_run checks its schedule and pointers before any CUDA call: these
    refusals need no GPU."""
    from paper_2307_12041_gb300.binding import Netlist, PlaceIterationArgs, PlaceSchedule
    nl = Netlist(1000, 300, None, None, None, None)
    a = PlaceIterationArgs(ctypes.pointer(nl), 1.0, 1.0, 64, 1, 0, 0, 1000)
    a.stats = 1 << 20
    good = dict(max_iters=100, tau_stop=0.1, bin_area=1.0 / 4096, area_mov=0.5, bin_w=1.0 / 64)
    fake = 1 << 20                                  # 16-byte aligned; refused before it is used

    def run(sched, state=fake, trace=fake):
        return L.pp_place_run(ctypes.byref(a), sched, state, trace, fake, 1 << 40, None)

    assert run(None) == 1
    for bad in (dict(max_iters=0), dict(max_iters=(1 << 24) + 1), dict(tau_stop=float("nan")),
                dict(bin_area=0.0), dict(area_mov=-1.0), dict(bin_w=float("inf"))):
        sc = PlaceSchedule(**dict(good, **bad))
        assert run(ctypes.byref(sc)) == 1, bad
        assert L.pp_last_error().decode() != ""
    sc = PlaceSchedule(**good)
    assert run(ctypes.byref(sc), state=None) == 1
    assert run(ctypes.byref(sc), state=fake + 8) == 1           # state must be 16-byte aligned
    assert run(ctypes.byref(sc), trace=None) == 1
    assert run(ctypes.byref(sc), trace=fake + 4) == 1           # trace must be 8-byte aligned
    assert L.pp_place_run(ctypes.byref(a), ctypes.byref(sc), fake, fake, fake, 256, None) == 2   # workspace


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes mirrors of pp_problem, pp_netlist, pp_place_iteration_args
    and the device loop's schedule, state and record have the header's size and field
    offsets (a C program compiled against include/pp.h prints them)."""
    import json
    import shutil
    import subprocess
    from paper_2307_12041_gb300.binding import (Netlist, PlaceIterationArgs, PlaceRecord, PlaceSchedule, PlaceState,
                                                Problem)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"pp_problem": Problem, "pp_netlist": Netlist, "pp_place_iteration_args": PlaceIterationArgs,
               "pp_place_schedule": PlaceSchedule, "pp_place_state": PlaceState, "pp_place_record": PlaceRecord}
    # the C names of the fields the binding renames
    c_name = {("pp_place_iteration_args", "lam"): "lambda", ("pp_place_state", "lam"): "lambda",
              ("pp_place_record", "lam"): "lambda"}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pp.h"', 'int main(void) {', 'printf("{");']
    first = True
    for sname, cls in mirrors.items():
        for fname, _ in cls._fields_:
            cf = c_name.get((sname, fname), fname)
            sep = "" if first else ","
            first = False
            lines.append(f'printf("{sep}\\"{sname}.{fname}\\": %zu", offsetof({sname}, {cf}));')
        lines.append(f'printf(",\\"{sname}.sizeof\\": %zu", sizeof({sname}));')
    lines += ['printf("}\\n");', "return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = json.loads(subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout)
    for sname, cls in mirrors.items():
        assert got[f"{sname}.sizeof"] == ctypes.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert got[f"{sname}.{fname}"] == getattr(cls, fname).offset, (sname, fname)


def test_host_workspace_adds_the_staging_arrays(L):
    for prec in (0, 1, 2):
        for n in (0, 1000, 12345):
            p = _prob(n=n)
            core = L.pp_workspace_size(ctypes.byref(p), prec)
            host = L.pp_grad_host_workspace_size(ctypes.byref(p), prec)
            per = ((4 * n + 255) // 256) * 256
            assert host == core + 256 + 8 * per, (prec, n)
    assert L.pp_grad_host_workspace_size(ctypes.byref(_prob(W=0.0)), 0) == 0
    assert L.pp_grad_host_workspace_size(ctypes.byref(_prob()), 7) == 0
