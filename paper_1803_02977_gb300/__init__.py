"""GB300-native (sm_103a) landscape-evolution time step of Barnes,
"Accelerating a Landscape Evolution Model with Parallelism" (arXiv:1803.02977).

The compute path is the CUDA library liblem.so behind the C ABI in
include/lem.h; `lem` is its ctypes binding and `synth` the seeded inputs.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "lem", "build"]
