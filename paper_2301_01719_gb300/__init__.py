"""GB300-native radiance-texture synthesis (Fober, arXiv 2301.01719, Section 2).

The compute path is libradtex, a C-ABI library of hand-written CUDA kernels
for sm_103a (include/radtex.h).  This package builds it (``build``), binds it
with the same entry-point names (``api``) and wraps forward/backward in a
``torch.autograd.Function`` (``autograd``).  Importing a submodule that calls
the library fails loudly when the library has not been built; there is no
other code path.
"""
import importlib

__all__ = ["api", "autograd", "build", "fit"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
