"""GB300 (sm_103a) tile rasterizer for 3D skew Gaussians.

Submodules:
  scenes      seeded synthetic inputs (no rasterizer arithmetic)
  build       nvcc build of libskewraster.so (in-tree)
  native      ctypes binding of the C ABI (include/skewraster.h)
  rasterizer  torch-facing API and autograd wrapper

Importing the package does not load CUDA; ``native.load()`` does.
"""

__all__ = ["scenes", "build", "native", "rasterizer"]
