"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and
the benchmark.  Holds none of the dual messenger arithmetic: spectra, noise
levels, masks and Gaussian draws only."""
from .generators import *  # noqa: F401,F403
