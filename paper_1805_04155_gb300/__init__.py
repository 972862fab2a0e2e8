"""GB300-native elastoplastic hot path: return mapping, tangent assembly and
Krylov-Newton load paths behind the C ABI of include/ep.h.

The compute path is the CUDA library libep.so (built by `build.build()`);
`ep` is its ctypes binding.  Importing `ep` requires the built library.
"""
from . import build  # noqa: F401
