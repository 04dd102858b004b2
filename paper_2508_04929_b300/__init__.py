"""B300-native (sm_103a) cryoSplat orthographic splatting path.

The compute path is libgs.so (hand-written CUDA behind the C-ABI of include/gs.h); the
Python modules bind it (``_lib``), sequence its calls over torch-allocated buffers
(``splat``), and build training machinery on top.  ``synth`` draws seeded synthetic inputs
and needs neither torch nor the library.  Submodules load lazily, so importing the package
does not load the CUDA library; using any compute entry point does, and raises if the
library is missing (there is no CPU fallback).
"""
import importlib

__all__ = ["synth", "build", "_lib", "splat"]


def __getattr__(name):
    if name in ("synth", "build", "_lib", "splat", "autograd", "batched", "autotune", "pointmlp"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
