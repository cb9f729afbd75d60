"""Counter-based random numbers of the descent driver, restated on the CPU
(TEST INFRASTRUCTURE ONLY: only the tests may import this module; it shares no
code with the CUDA library, which implements the same published definitions).

The descent loop (a stand-in for the placer loop of Sec. IV, whose parameters
the paper does not give) perturbs every block by a seed-fixed jitter.  The jitter
cannot be passed in for 10^7 blocks and 100 steps without dominating the step,
so both sides draw it from one counter-based generator:

* Philox4x32-10 (J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel
  random numbers: as easy as 1, 2, 3", SC 2011): a 4 x 32-bit counter and a
  2 x 32-bit key, ten rounds of two 32 x 32 -> 64-bit products with the
  multipliers 0xD2511F53 and 0xCD9E8D57, the key bumped by the Weyl constants
  0x9E3779B9 and 0xBB67AE85 after each round.
* Box-Muller: for uniforms u0 in (0, 1], u1 in [0, 1), r = sqrt(-2 ln u0),
  (n0, n1) = r (cos 2 pi u1, sin 2 pi u1) are two independent standard normals.

Block i at step k uses counter (i, k, 0, 0) and key (seed mod 2^32, seed >> 32);
u0 = (out0 + 1/2) 2^-32, u1 = (out1 + 1/2) 2^-32; the x jitter is n0, the y jitter n1.
"""
from __future__ import annotations

import numpy as np

M32 = np.uint64(0xFFFFFFFF)
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85


def philox4x32_10(ctr, key):
    """ctr: (4, n) uint32-valued array (or 4 ints), key: (k0, k1) ints -> (4, n) uint64."""
    c = [np.asarray(v, dtype=np.uint64) & M32 for v in ctr]
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for _ in range(10):
        p0 = PHILOX_M0 * c[0]
        p1 = PHILOX_M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & M32
        hi1, lo1 = p1 >> np.uint64(32), p1 & M32
        c = [(hi1 ^ c[1] ^ np.uint64(k0)) & M32, lo1, (hi0 ^ c[3] ^ np.uint64(k1)) & M32, lo0]
        k0 = (k0 + PHILOX_W0) & 0xFFFFFFFF
        k1 = (k1 + PHILOX_W1) & 0xFFFFFFFF
    return np.stack(c)


def box_muller(out0, out1):
    u0 = (np.asarray(out0, dtype=np.float64) + 0.5) * 2.0 ** -32
    u1 = (np.asarray(out1, dtype=np.float64) + 0.5) * 2.0 ** -32
    r = np.sqrt(-2.0 * np.log(u0))
    return r * np.cos(2.0 * np.pi * u1), r * np.sin(2.0 * np.pi * u1)


def descent_normals(n: int, seed: int, step: int, idx=None):
    """(2, len(idx)) standard normals of blocks idx (default all n) at `step`."""
    i = np.arange(n, dtype=np.uint64) if idx is None else np.asarray(idx, dtype=np.uint64)
    z = np.zeros_like(i)
    out = philox4x32_10([i, np.full_like(i, step), z, z], (seed & 0xFFFFFFFF, seed >> 32))
    n0, n1 = box_muller(out[0], out[1])
    return np.stack([n0, n1])


def descent_step(W, H, x, y, w, h, gx, gy, movable, lr, sigma, seed, step):
    """The position update of the descent loop, in float64 (see descent_normals):
    x <- clip(x - lr gx + sigma n0, w/2, W - w/2), likewise y; fixed blocks stay."""
    x, y, w, h, gx, gy = (np.asarray(v, dtype=np.float64) for v in (x, y, w, h, gx, gy))
    nrm = descent_normals(len(x), seed, step)
    xn = np.clip(x - lr * gx + sigma * nrm[0], w / 2, W - w / 2)
    yn = np.clip(y - lr * gy + sigma * nrm[1], h / 2, H - h / 2)
    if movable is not None:
        mv = np.asarray(movable, dtype=bool)
        xn = np.where(mv, xn, x)
        yn = np.where(mv, yn, y)
    return xn, yn
