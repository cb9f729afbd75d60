"""FP64 check of a saved descent run against the oracle (test infrastructure).

The descent CLI (python -m paper_2307_12041_gb300.descent ... --save-dir DIR)
writes DIR/stepKKK.npz for its first and last steps: the GPU's gradient and
per-block energy on a seeded sample of blocks and its total energy E, and for the
last step every block's position as ulp steps from its start.  This script
rebuilds the positions (the start is the seeded workload), evaluates the oracle's
full FP64 coefficients of the whole placement at each saved step, and prints the
sample's max / RMS errors of the gradient and N and the relative error of E, as
one JSON line per step.

  python tests/check_descent_against_oracle.py DIR [--workload 4] [--n N]
"""
import argparse
import glob
import json
import lzma
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import series as O                     # noqa: E402
from paper_2307_12041_gb300 import synth           # noqa: E402


def positions(start, rec, name):
    k = np.frombuffer(lzma.decompress(rec[name].tobytes()), dtype=np.dtype(str(rec[name + "_dtype"])))
    x = np.asarray(start, np.float32).astype(np.float64) + k.astype(np.float64) * 0.5 * np.spacing(
        np.abs(np.asarray(start, np.float32))).astype(np.float64)
    x32 = x.astype(np.float32)
    assert np.array_equal(x32.astype(np.float64), x), "positions do not reconstruct exactly"
    return x32


def energy_from_coeffs(a, W, H):
    Mx, My = a.shape
    eu = np.where(np.arange(Mx) == 0, 1.0, 2.0)
    ev = np.where(np.arange(My) == 0, 1.0, 2.0)
    k2 = (np.arange(Mx)[:, None] * math.pi / W) ** 2 + (np.arange(My)[None, :] * math.pi / H) ** 2
    k2[0, 0] = 1.0
    G = eu[:, None] * ev[None, :] / (W * H * k2)
    G[0, 0] = 0.0
    S = np.where(G > 0, a / np.where(G > 0, G, 1.0), 0.0)
    return 0.5 * float(np.sum(a * S))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("dir")
    ap.add_argument("--workload", type=int, default=4)
    ap.add_argument("--n", type=int, default=None, help="first n blocks (as the descent's --n)")
    ap.add_argument("--modes", type=int, default=None, help="modes per axis if not the workload's")
    args = ap.parse_args(argv)
    p = synth.workload(args.workload, n=args.n)
    if args.modes:
        p.Mx = p.My = args.modes
    for path in sorted(glob.glob(os.path.join(args.dir, "step*.npz"))):
        rec = np.load(path)
        x, y = p.x, p.y
        if "dx" in rec:
            x, y = positions(p.x, rec, "dx"), positions(p.y, rec, "dy")
        idx = rec["sample"]
        t0 = time.time()
        a = O.coefficients(p.W, p.H, x, y, p.w, p.h, p.c, p.Mx, p.My)
        N, gx, gy = O.energy_grad(p.W, p.H, x, y, p.w, p.h, p.c, a, idx=idx)
        E = energy_from_coeffs(a, p.W, p.H)
        scale = max(np.max(np.abs(gx)), np.max(np.abs(gy)))
        dg = np.concatenate([rec["gx"] - gx, rec["gy"] - gy])
        out = {"step": int(rec["step"]), "n": int(p.n), "Mx": p.Mx, "My": p.My, "sample": int(len(idx)),
               "grad_max": float(np.max(np.abs(dg)) / scale),
               "grad_rms": float(np.sqrt(np.mean(dg ** 2)) / np.sqrt(np.mean(np.concatenate([gx, gy]) ** 2))),
               "N_max": float(np.max(np.abs(rec["N"] - N)) / np.max(np.abs(N))),
               "N_rms": float(np.sqrt(np.mean((rec["N"] - N) ** 2)) / np.sqrt(np.mean(N ** 2))),
               "E_gpu": float(rec["E"]), "E_oracle": E, "E_rel": abs(float(rec["E"]) - E) / abs(E),
               "oracle_s": time.time() - t0, "threads": O._threads()}
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
