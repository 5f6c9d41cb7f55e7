"""GB300-native meta-estimated inverse path tracing (arXiv 2309.15676 hot path).

The compute path is the CUDA library built from csrc/ (C ABI in include/mer.h);
`api` and `autograd` only marshal arguments to it. `synth` builds seeded inputs.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "api", "autograd", "build"]
