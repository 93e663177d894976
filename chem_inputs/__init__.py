"""Seeded input generators shared by the oracle and the GPU path.

Data only: the synthetic mechanism (``mechanism``) and the cell-state recipes
(``workloads``).  Nothing here evaluates the chemistry or the integrator.
"""
from . import mechanism, workloads  # noqa: F401
