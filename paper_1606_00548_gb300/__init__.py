"""GB300-native fully implicit reservoir Newton step (arXiv:1606.00548 hot path).

    synth   seeded synthetic inputs (grid, rock, fluids, wells)
    build   nvcc build of libsim.so (sm_103a)
    sim     ctypes binding of the C ABI in include/sim.h
"""
from . import synth  # noqa: F401

__all__ = ["synth", "build", "sim"]
