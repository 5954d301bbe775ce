"""GB300-native Sparse Bessel Decomposition (arXiv:1711.07877): the on-line SBD matvec.

The computation lives in libsbd.so (hand-written CUDA for sm_103a plus a host
off-line plan in C++); the ``sbd`` submodule is its ctypes binding, whose names
are re-exported here on first use.  Using any of them fails loudly (ImportError)
when the library has not been built (python -m paper_1711_07877_gb300.build);
there is no fallback.
"""
import importlib
import os

_SUBMODULES = {name[:-3] for name in os.listdir(os.path.dirname(__file__)) if name.endswith(".py")}


def __getattr__(name):
    if name.startswith("__"):
        raise AttributeError(name)
    if name in _SUBMODULES:
        return importlib.import_module(f"{__name__}.{name}")
    mod = importlib.import_module(__name__ + ".sbd")   # loads libsbd.so
    try:
        return getattr(mod, name)
    except AttributeError:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from None
