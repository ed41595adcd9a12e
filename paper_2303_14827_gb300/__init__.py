"""GB300-native renderer for dual-quaternion Julia isosurfaces (Kenwright,
"Dual-Quaternion Julia Fractals").

The compute path is a hand-written sm_103a CUDA library (``libdqj.so``) behind a
C ABI declared in ``include/dqj.h``; ``binding`` is a thin ctypes layer with the
same names.  Importing this package loads nothing: the library is loaded on first
use, and a missing library is an error, never a fallback.
"""
__all__ = ["scenes"]
