"""Phase step of the basis generators (the cos/sin factors of Eq. aup) against
exact arithmetic: s = x * (1/L) is formed exactly from the float32 x and the
double 1/L as the records form it, reduced modulo 2 and rounded to 2^-62
half-turns with Python integers, m*s mod 2 is taken
exactly, and cos/sin of pi times that phase come from FP64 numpy.  Both device
evaluators (the sincospif-based one of the records and CUDA-core kernels, and the
Taylor-polynomial anchor of the BF16x3 generators) must agree to a few FP32 units
at every mode up to 65535, including phases that need exact reduction (m * s far
beyond FP32's reach).  The TF32 generators' anchor (the hardware sine and cosine
of the exactly reduced phase) must stay within its documented bound: absolute
error at most 2^-21.41 (3.6e-7) for arguments in [-pi, pi], plus the rounding of
the 31-bit phase to FP32 (2^-24 of pi, 1.9e-7) and of the product by pi (1e-7):
1e-6 in all."""
import math
from fractions import Fraction

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def exact_phase(x32, L, m):
    """(cos, sin)(pi * (m * s mod 2)) with s = x * fl64(1/L) (exact product of the
    float32 x and the double 1/L) reduced mod 2 and rounded to 2^-62 half-turns."""
    out = np.empty((len(x32), 2))
    invL = Fraction(1.0 / L)
    for i, (xv, mv) in enumerate(zip(x32, m)):
        v = Fraction(float(xv)) * invL * 2 ** 62          # exact, in 2^-62 half-turn units
        f = math.floor(abs(v) + Fraction(1, 2))           # nearest, ties away from zero
        f = (-f if v < 0 else f) % 2 ** 63                # reduced mod 2 half-turns
        p = (int(mv) * f) % 2 ** 63                      # m s mod 2, exact
        th = math.pi * (p / 2 ** 62)
        out[i] = (math.cos(th), math.sin(th))
    return out


def cases(seed, n, L):
    g = np.random.default_rng(seed)
    x = np.concatenate([g.uniform(0, L, n - 8), [0.0, L, 0.5 * L, 1e-7, L - 1e-7, 2.5 * L, 0.25 * L,
                                                 0.123456789 * L]]).astype(np.float32)
    m = np.concatenate([g.integers(0, 4097, n // 2), g.integers(0, 65536, n - n // 2 - 8),
                        [0, 1, 2, 4095, 4096, 65535, 1024, 3]]).astype(np.int32)
    return x, m


TOL = {0: 3e-7, 1: 3e-7, 2: 1e-6}


@pytest.mark.parametrize("L", [1.0, 0.7, 123.25])
@pytest.mark.parametrize("evaluator", [0, 1, 2])
def test_phase_evaluators_match_exact_reduction(pp, L, evaluator):
    x, m = cases(int(L * 100) + evaluator, 4000, L)
    got = pp.binding.phase_eval(torch.from_numpy(x).cuda(), L, torch.from_numpy(m).cuda(),
                                evaluator).double().cpu().numpy()
    ref = exact_phase(x, L, m)
    err = np.abs(got - ref).max()
    assert err <= TOL[evaluator], (evaluator, err)
    # unit modulus to FP32 rounding (to the hardware functions' error for evaluator 2)
    assert np.abs(np.hypot(got[:, 0], got[:, 1]) - 1).max() <= TOL[evaluator]


def test_phase_eval_rejects_bad_arguments(pp):
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    m = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(pp.binding.PPError):
        pp.binding.phase_eval(x, 0.0, m)
    with pytest.raises(pp.binding.PPError):
        pp.binding.phase_eval(x, 1.0, m, evaluator=3)
