"""GB300 (sm_103a) library for ABFT-protected 3D stencil sweeps (arXiv 1909.00709).

The compute path is the CUDA library ``libabft.so`` (C ABI in ``include/abft.h``),
reached through the ctypes binding in ``abi``.  ``inputs`` generates seeded
synthetic workloads; ``replicas`` holds the host logic of one process per GPU.  Submodules load lazily so that input generation works
without a GPU or a built library.
"""
import importlib

__all__ = ["abi", "inputs", "build", "replicas"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
