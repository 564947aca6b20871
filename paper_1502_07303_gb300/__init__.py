"""GB300-native restarted narrow band fast marching (Yang & Stern).

The compute path lives in the CUDA library ``libfmm_gb300.so`` (sources in
``csrc/``, C ABI in ``include/fmm.h``).  ``fmm`` is its thin ctypes binding and
``workloads`` the seeded input generators.  Submodules are imported lazily so
that importing the input generators never loads the CUDA library.
"""
import importlib

__all__ = ["fmm", "workloads", "build"]


def __getattr__(name):
    if name in ("fmm", "workloads", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
