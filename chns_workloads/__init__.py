"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

Only input generation lives here (octree leaf lists from refinement predicates, 2:1 balance,
closed-form initial fields). None of the finite-element arithmetic of the method does.
"""
from . import configs, fields, octree  # noqa: F401
from .octree import MAXD  # noqa: F401
