"""Seeded synthetic inputs (programs and fields) shared by the oracle and the
CUDA library's tests and benchmark.  Nothing in this package evaluates the
tiling method; see `synth.program` for the interchange format."""
from . import rng, program, workloads  # noqa: F401
