"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package produces the bytes both sides consume (random SU(3) gauge fields, APE
smearing, Gaussian and point sources, and the five workload descriptions).  It holds
none of the solver's arithmetic: no Dirac operator, no clover term, no Schwarz or
Krylov step.  Random numbers come from numpy's PCG64 so that every machine draws the
same stream for a given seed.
"""
from .gauge import random_su3_field, ape_smear, reunitarize, unit_gauge
from .sources import gaussian_source, point_sources
from .configs import WORKLOADS, Workload, make_gauge, make_sources

__all__ = [
    "random_su3_field", "ape_smear", "reunitarize", "unit_gauge",
    "gaussian_source", "point_sources", "WORKLOADS", "Workload",
    "make_gauge", "make_sources",
]
