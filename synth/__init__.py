"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the benchmark and the CPU oracle's
callers. It builds *data* only: prestack gathers with Ricker reflection
events and Gaussian noise, the acquisition geometry, the list of zero-offset
domains and their apertures. It evaluates no coherence, runs no search and
draws none of the random numbers the search itself uses.
"""
from .gathers import (  # noqa: F401
    Line, Problem, make_line, cmp_problem, line_problem, batched_problems, slab_bounds,
    slab_problem,
    crs_recentre, CMP, CRS,
)
from . import configs  # noqa: F401
