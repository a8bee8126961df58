"""B300-native direct N-body block-step Hermite integrator (libnb + binding).

The compute path is libnb.so (CUDA, sm_103a) behind the C ABI in include/nb.h;
`paper_1312_1789_b300.nb` is its ctypes binding.  Importing the package does not
load the library; `nb.lib()` does, and fails loudly if it is missing.
"""
__all__ = ["nb", "ics", "build"]
