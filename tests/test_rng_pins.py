"""Pins of the descent driver's counter-based generator (oracle/rng.py).

Philox4x32-10 against the known-answer vectors published with its definition
(Salmon et al., SC 2011, Random123): counter 0 / key 0, all-ones counter and
key, and the digits-of-pi counter and key.  Box-Muller normals: moments and
independence on 200,000 draws, and the closed form at known uniforms."""
import numpy as np

from oracle import rng

KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


def test_philox_known_answers():
    for ctr, key, want in KAT:
        got = rng.philox4x32_10([[v] for v in ctr], key)[:, 0]
        assert [int(v) for v in got] == list(want)


def test_philox_vectorised_matches_scalar():
    i = np.arange(50, dtype=np.uint64)
    z = np.zeros_like(i)
    out = rng.philox4x32_10([i, np.full_like(i, 7), z, z], (123, 456))
    for j in (0, 17, 49):
        one = rng.philox4x32_10([[j], [7], [0], [0]], (123, 456))[:, 0]
        assert np.array_equal(out[:, j], one)


def test_box_muller_closed_form():
    # u0 = 1/4 (out0 = 2^30 - 1/2 cannot be hit; use the formula's inputs directly)
    n0, n1 = rng.box_muller([2 ** 31 - 0.5], [2 ** 30 - 0.5])     # u0 = 1/2, u1 = 1/4
    r = np.sqrt(-2 * np.log(0.5))
    assert abs(n0[0] - 0.0) < 1e-12 * r + 1e-15 and abs(n1[0] - r) < 1e-12


def test_normals_moments_and_independence():
    nrm = rng.descent_normals(200_000, seed=2307_12041, step=3)
    for row in nrm:
        assert abs(row.mean()) < 0.01 and abs(row.var() - 1) < 0.01
        assert abs(np.mean(row ** 4) - 3) < 0.06                   # Gaussian kurtosis
    assert abs(np.corrcoef(nrm)[0, 1]) < 0.01
    other = rng.descent_normals(200_000, seed=2307_12041, step=4)
    assert abs(np.corrcoef(nrm[0], other[0])[0, 1]) < 0.01       # steps are independent
