"""Writes uniform-2k-64x64.json: oracle values on the seeded 2,000-block 64 x 64
workload (E in both readings, sampled coefficients, sampled per-block energies
and gradients).  The paper prints no worked example (its figures are absent from
the text), so this fixture is a regression record of the FP64 oracle, written only
by this script from oracle/ and the input generator:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import series as O                      # noqa: E402
from paper_2307_12041_gb300 import synth            # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "uniform-2k-64x64.json")


def compute():
    p = synth.workload(0)
    g = np.random.default_rng(20230722)
    modes = [(int(u), int(v)) for u, v in zip(g.integers(0, p.Mx, 40), g.integers(0, p.My, 40))]
    blocks = sorted(int(i) for i in g.choice(p.n, 40, replace=False))
    a = O.coefficients(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    N, gx, gy = O.energy_grad(p.W, p.H, p.x, p.y, p.w, p.h, p.c, a)
    Nc = O.energy_grad(p.W, p.H, p.x, p.y, p.w, p.h, p.c, a, sample="center")[0]
    return {
        "workload": synth.WORKLOADS[0]["name"], "n": p.n, "Mx": p.Mx, "My": p.My,
        "E_rect": 0.5 * float(N.sum()), "E_center": 0.5 * float(Nc.sum()),
        "modes": modes, "a": [float(a[u, v]) for u, v in modes],
        "blocks": blocks, "N": [float(N[i]) for i in blocks],
        "gx": [float(gx[i]) for i in blocks], "gy": [float(gy[i]) for i in blocks],
        "a_max": float(np.abs(a).max()), "N_max": float(np.abs(N).max()),
        "g_max": float(max(np.abs(gx).max(), np.abs(gy).max())),
    }


if __name__ == "__main__":
    with open(OUT, "w") as fh:
        json.dump(compute(), fh, indent=1)
    print("wrote", OUT)
