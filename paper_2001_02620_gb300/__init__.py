"""qrt: a GB300-native two-level quad-BVH ray tracer and path tracer.

Layout:
  csrc/        CUDA kernels (traversal, path tracer, adjoint), host BVH
               builder and the C ABI declared in include/qrt.h
  _native.py   ctypes declarations of the C ABI (same names)
  api.py       Scene / RenderGraph / RenderFn on top of PyTorch tensors
  inputs.py    seeded synthetic workloads (shared with the test oracle)
  autotune.py  launch-parameter search with a JSON cache
  shard.py     image-parallel tile sharding across ranks
  build.py     in-tree build of libqrt.so for sm_103a

Submodules are imported lazily so that importing the input generator does not
load the CUDA library.
"""
import importlib

__all__ = ["api", "inputs", "autotune", "shard", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
