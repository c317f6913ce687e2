"""GB300 (sm_103a) RBF-FD solution of Poisson's equation on scattered nodes.

The compute path is the C-ABI library librbffd.so (include/rbffd.h), built
from csrc/ by `_build.build()`; `rbffd` binds it with ctypes and `pipeline`
composes the calls.  Importing the package does not touch the GPU; the
first binding call loads the library and raises if it is missing or fails.
"""

from . import _build  # noqa: F401

__all__ = ["rbffd", "pipeline"]


def __getattr__(name):
    if name in ("rbffd", "pipeline"):
        import importlib

        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
