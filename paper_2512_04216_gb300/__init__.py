"""GB300 state-vector simulation: the C-ABI library libsvgb.so and its binding.

``capi`` mirrors include/sv.h one function per entry point; ``StateVector``
is a small convenience object over it that takes device memory and streams
from PyTorch.  Using either requires the built library (see
``paper_2512_04216_gb300.build``): loading ``capi`` raises ImportError when it
is missing -- there is no CPU fallback.  The submodules load on first use so
that the build script can run before the library exists.
"""
import importlib

__all__ = ["capi", "StateVector", "Batch", "build"]


def __getattr__(name):
    if name in ("capi", "build", "statevector", "batch", "serve", "costmodel"):
        return importlib.import_module(f".{name}", __name__)
    if name == "StateVector":
        return importlib.import_module(".statevector", __name__).StateVector
    if name == "Batch":
        return importlib.import_module(".batch", __name__).Batch
    raise AttributeError(name)
