"""Failure path on the GPU without a fault: a kernel's bounded wait on an
mbarrier that nothing completes runs out, the kernel records the timeout in the
device status word and returns; the host reads PP_ETIMEOUT, the word is cleared,
and the same context then evaluates correctly."""
import time

import numpy as np
import pytest

from oracle import series as O
from paper_2307_12041_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("limit_ms", [1, 50])
def test_bounded_wait_runs_out_and_is_reported(pp, limit_ms):
    pp.binding.sync_status()                         # start from a clear status word
    t0 = time.perf_counter()
    pp.binding.check_wait_timeout(limit_ms * 1_000_000)
    with pytest.raises(pp.binding.PPError) as err:
        pp.binding.sync_status()
    elapsed = time.perf_counter() - t0
    assert err.value.status == 4                     # PP_ETIMEOUT
    assert elapsed >= 0.9 * limit_ms / 1e3
    assert elapsed < 5.0
    pp.binding.sync_status()                         # read and cleared: no error now


def test_context_usable_after_timeout(pp):
    pp.binding.check_wait_timeout(10_000_000)
    with pytest.raises(pp.binding.PPError):
        pp.binding.sync_status()
    p = synth.uniform_blocks(700, 40, 48, seed=17)
    ref = O.evaluate(p.W, p.H, p.x, p.y, p.w, p.h, p.c, p.Mx, p.My)
    for prec in pp.binding.available_precisions():
        out = pp.binding.evaluate(p, prec=prec)
        pp.binding.sync_status()
        a = out["a"].double().cpu().numpy()
        assert np.max(np.abs(a - ref["a"])) <= pp.binding.TOLERANCE[prec] * np.max(np.abs(ref["a"]))
        N = out["N"].double().cpu().numpy()
        assert np.max(np.abs(N - ref["N"])) <= pp.binding.TOLERANCE[prec] * np.max(np.abs(ref["N"]))
