"""GB300-native flux-reconstruction (FR) right-hand-side engine.

The compute path lives in libfr.so (CUDA kernels for sm_103a behind the C
ABI of include/fr.h); `fr` is its ctypes binding and `build` compiles it.
"""
__all__ = ["fr", "build"]
