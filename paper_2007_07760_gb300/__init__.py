"""GB300-native DUGKS time step for the conservative Allen-Cahn equation.

The compute path is libdugks.so (hand-written sm_103a CUDA behind a C ABI,
include/dugks.h); ``native`` is its ctypes binding and ``workloads`` builds the
seeded synthetic inputs.
"""
from . import workloads  # noqa: F401

__all__ = ["native", "workloads"]
