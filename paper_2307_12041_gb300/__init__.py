"""GB300-native analytical Poisson series for placement density (arXiv 2307.12041).

The compute path is the C-ABI CUDA library `libpp.so` (built in-tree by
`__graft_entry__.build()`); `binding` marshals torch tensors into its calls.
Importing this package does not load the library; `load()` does, and every
compute call fails loudly if it is missing.
"""
import importlib

from . import synth  # noqa: F401

_BINDING_NAMES = ("coeffs", "energy", "grad", "evaluate", "PoissonEnergy", "Problem",
                  "workspace", "sync_status", "PRECISIONS", "SAMPLES", "PPError")


def load():
    return importlib.import_module(__name__ + ".binding").lib()


def __getattr__(name):
    if name in ("binding", "build_lib", "descent"):
        return importlib.import_module(__name__ + "." + name)
    if name in _BINDING_NAMES:
        return getattr(importlib.import_module(__name__ + ".binding"), name)
    raise AttributeError(name)
