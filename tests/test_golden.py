"""The oracle still reproduces its recorded values on the 2,000-block 64 x 64
workload (tests/golden/, written by tests/golden/make_golden.py), and the CUDA
path matches them within each precision's tolerance."""
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden", "uniform-2k-64x64.json")


def load():
    with open(GOLD) as fh:
        return json.load(fh)


def test_oracle_reproduces_golden():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden",
                                                  os.path.join(os.path.dirname(GOLD), "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    now, gold = mg.compute(), load()
    for k in ("E_rect", "E_center"):
        assert abs(now[k] - gold[k]) <= 1e-12 * abs(gold[k])
    for k in ("a", "N", "gx", "gy"):
        assert np.allclose(now[k], gold[k], rtol=1e-11, atol=1e-300)


@pytest.mark.gpu
def test_cuda_path_matches_golden(pp):
    from paper_2307_12041_gb300 import synth
    gold = load()
    p = synth.workload(0)
    for prec in pp.binding.available_precisions():
        tol = pp.binding.TOLERANCE[prec]
        out = pp.binding.evaluate(p, prec=prec)
        a = out["a"].double().cpu().numpy()
        got = np.array([a[u, v] for u, v in gold["modes"]])
        assert np.max(np.abs(got - gold["a"])) <= tol * gold["a_max"], prec
        for k, scale in (("N", "N_max"), ("gx", "g_max"), ("gy", "g_max")):
            v = out[k].double().cpu().numpy()[gold["blocks"]]
            assert np.max(np.abs(v - gold[k])) <= tol * gold[scale], (prec, k)
        assert abs(out["E"] - gold["E_rect"]) <= tol * abs(gold["E_rect"]), prec
