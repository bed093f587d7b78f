"""GB300-native detector-error-model compiler (GreenPeas two-stage error analysis).

Submodules:
  circuits  circuit IR and seeded workload generators (inputs only)
  build     nvcc build of the sm_103a library
  native    ctypes declarations of the C ABI (include/gpdem.h)
  dem       Driver / Dem / DemFunction over the C ABI
"""
__all__ = ["circuits", "build", "native", "dem"]


def __getattr__(name):
    import importlib
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
