"""GB300-native (sm_103a) application of sequences of planar rotations.

Method: Steel & Langou, "Communication efficient application of sequences of
planar rotations to a matrix".  The computation runs in the CUDA library built
from ``csrc/`` (C ABI: ``include/rotseq.h``); this package holds its Python
binding (``api``), the seeded workload generators (``workloads``) and the build
script (``build``).  The binding is imported on first use so that the
generators can be used without torch or a GPU.
"""
__all__ = ["rot_apply", "rot_apply_f32", "rot_device_status", "colmajor", "empty_colmajor",
           "RotError"]


def __getattr__(name):
    if name in __all__:
        from . import api, _native
        if name == "RotError":
            return _native.RotError
        return getattr(api, name)
    raise AttributeError(name)
