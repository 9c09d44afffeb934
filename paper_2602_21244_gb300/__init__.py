"""GB300 (sm_103a) DSMC collision step of arXiv 2602.21244.

``paper_2602_21244_gb300.dsmc`` is the ctypes binding of the CUDA library
(``libdsmc.so``, C ABI in ``include/dsmc.h``); ``workloads`` draws the
seeded synthetic gases.  Importing ``dsmc`` builds the library if needed and
raises if it cannot be built or loaded: there is no CPU fallback.
"""
import importlib

__all__ = ["dsmc", "workloads"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
