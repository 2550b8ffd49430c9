"""GB300-native dynamic-graph random walks (FlowWalker, arXiv 2404.08364).

The compute path is libfw.so (hand-written sm_103a CUDA behind the C ABI in
include/fw.h); this package holds its build script and a thin torch-facing
binding.  Importing the package does not load the library; the first use of
``DeviceGraph`` does, and raises if it is missing.
"""

__all__ = ["DeviceGraph", "Server", "sample", "build"]


def build(force: bool = False) -> str:
    from .build import build as _b
    return _b(force=force)


def __getattr__(name):
    if name in ("DeviceGraph", "Server", "sample"):
        from . import walker
        return getattr(walker, name)
    raise AttributeError(name)
