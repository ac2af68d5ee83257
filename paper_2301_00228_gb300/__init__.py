"""GB300-native plane-strain lattice Boltzmann solver (arXiv:2301.00228).

The time loop runs in hand-written sm_103a CUDA kernels behind the C-ABI of
``include/lbps.h``; ``paper_2301_00228_gb300.lbps`` is the thin ctypes binding
with the same names.  ``workloads`` draws seeded synthetic inputs.  Submodules
are imported on use so that importing the package needs neither a GPU nor the
compiled library.
"""
import importlib

__all__ = ["lbps", "workloads"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
