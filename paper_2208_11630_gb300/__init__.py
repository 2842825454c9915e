"""GB300-native (sm_103a) block-AMR compressible Euler hot path.

The CUDA kernels sit behind the C ABI in ``include/fx.h`` (``libfx.so``);
``fx`` is the thin Python binding (it loads the library on first use),
``inputs`` the seeded synthetic inputs.
"""
from . import fx, inputs  # noqa: F401

__all__ = ["inputs", "fx"]
