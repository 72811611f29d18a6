"""Seeded synthetic lattice fields (gauge links, spinors, gauge transforms).

Shared by the CPU oracle's tests and the CUDA path's tests and benchmark as
input data only: nothing here applies the Wilson-Dirac operator.
"""
from . import rng, fields  # noqa: F401
