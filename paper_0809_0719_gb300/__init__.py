"""GB300 butterfly algorithm for discrete Fourier integral operators
(Candes, Demanet & Ying 2008).

The compute path is the CUDA library libfio.so (C ABI in include/fio.h); the
Python modules only marshal arguments (fio), build the library (build) and draw
seeded synthetic inputs (inputs).  Submodules load lazily so that importing the
package never touches the GPU.
"""
__all__ = ["fio", "build", "inputs"]


def __getattr__(name):
    if name in __all__:
        import importlib

        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
