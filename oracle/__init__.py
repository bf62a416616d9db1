"""CPU FP64 oracle for the 2D (dbi_oracle) and 3D (dbi_oracle3d, as `o3d`) elastic
Lippmann-Schwinger operators and the distorted-Born products built on them.

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
It shares no code with the CUDA library and imports nothing from it.
"""
from .dbi_oracle import *  # noqa: F401,F403
from .dbi_oracle import LSOracle, normalized_error  # noqa: F401
from . import dbi_oracle3d as o3d  # noqa: F401
