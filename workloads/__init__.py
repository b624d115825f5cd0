"""Seeded synthetic input generators shared by the oracle tests, the GPU tests and the benchmark.

This package holds no arithmetic of the streaming Tucker method itself: it only draws random
numbers and evaluates the closed-form synthetic fields described in the module docstrings.
Every tensor it returns is laid out column-major (mode 1 fastest), the matricization convention
of the paper (Sec. 2.1).
"""

from .synth import (  # noqa: F401
    LowRankStream,
    BlobField,
    SineWave,
    random_orthonormal,
    config1_tensor,
    CONFIG1,
    CONFIG2,
    CONFIG5,
    batched_streams,
)
