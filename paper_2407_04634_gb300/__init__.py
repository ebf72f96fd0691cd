"""GB300-native randomized small-block Lanczos null-space solver.

The compute path is the CUDA library libnullspace.so (C ABI in
include/nullspace.h); `nullspace` is its thin ctypes binding.  Importing this
package does not load the library; call `nullspace.load()` (done on first use).
"""

__all__ = ["nullspace", "build"]
