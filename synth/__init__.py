"""Seeded synthetic inputs (scenes, scans, poses) shared by the oracle tests,
the CUDA parity tests and the benchmark.  Holds no mapping arithmetic."""
from .scenes import *  # noqa: F401,F403
