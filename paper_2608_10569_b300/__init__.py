"""B300-native HWENO-GR solver for the 2D compressible Navier-Stokes equations.

The compute path is the CUDA library ``libhweno.so`` behind the C ABI in
``include/hweno.h``; ``paper_2608_10569_b300.hweno`` is its thin ctypes binding.
Submodules load lazily so that ``inputs`` can be used without a GPU.
"""
__all__ = ["inputs", "hweno"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
