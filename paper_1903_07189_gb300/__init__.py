"""GB300 (sm_103a) implementation of the Weighted Mean Curvature (WMC) stencil and the
WMC-regularised image flows of Gong & Goksel, arXiv 1903.07189.

The compute path is ``libwmc.so`` (CUDA C++, C ABI in include/wmc.h).  ``wmc`` is its Python
binding; ``synth`` makes seeded synthetic test images.  The binding is imported lazily so
that the generator can be used without a GPU or a built library.
"""
import importlib

__all__ = ["wmc", "synth", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
