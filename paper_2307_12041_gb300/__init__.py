"""GB300-native analytical Poisson series for placement density (arXiv 2307.12041).

The compute path is the C-ABI CUDA library `libpp` (built in-tree by
`__graft_entry__.build()`); `binding` marshals torch tensors into its calls.
Importing this package does not load the library; `load()` does, and every
compute call fails loudly if it is missing.
"""
from . import synth  # noqa: F401


def load():
    from . import binding
    return binding.lib()


def __getattr__(name):
    if name in ("coeffs", "energy", "grad", "energy_grad", "PoissonEnergy", "Problem",
                "workspace_size", "sync_status", "Precision", "Sample", "PPError", "binding"):
        from . import binding
        return getattr(binding, name)
    raise AttributeError(name)
