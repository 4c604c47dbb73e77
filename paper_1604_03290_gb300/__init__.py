"""GB300-native solid-body SPH right-hand side (Schaefer et al. 2016).

``sph``        ctypes binding of the CUDA library ``libsph.so`` (include/sph.h)
``workloads``  seeded synthetic particle sets shaped like the paper's tests
``build``      in-tree nvcc build of the library for sm_103a
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "sph", "build"]


def __getattr__(name):
    if name in ("sph", "build"):
        import importlib
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
