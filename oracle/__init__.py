"""FP64 CPU oracle of the analytical Poisson series (test infrastructure only).

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import this package.  It shares no code with the CUDA library.
"""
from .series import (coefficients, energy_grad, evaluate, field, potential,  # noqa: F401
                     rect_integrals, sine_differences, cosine_differences, total_energy)
