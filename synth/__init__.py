"""Seeded synthetic inputs (shapes, boundary samples, query points, rotations, poses).

Shared by the CUDA path's tests and benchmark and by the CPU oracle.  Holds no
arithmetic of the method itself.
"""
from . import configs, rotations, shapes  # noqa: F401
