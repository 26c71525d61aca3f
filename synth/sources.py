"""Seeded spinor sources (input generation only).

A spinor is complex128 of shape (Lt, Lz, Ly, Lx, 4, 3): [t, z, y, x, spin, colour].
"""
from __future__ import annotations

import numpy as np


def gaussian_source(dims, seed: int) -> np.ndarray:
    """Every real component ~ N(0, 1), drawn with PCG64(seed) in (re, im) order."""
    Lx, Ly, Lz, Lt = dims
    g = np.random.Generator(np.random.PCG64(seed)).standard_normal(size=(Lt, Lz, Ly, Lx, 4, 3, 2))
    return g[..., 0] + 1j * g[..., 1]


def point_sources(dims) -> list[np.ndarray]:
    """The 12 unit vectors at site 0, one per (spin, colour)."""
    Lx, Ly, Lz, Lt = dims
    out = []
    for s in range(4):
        for c in range(3):
            v = np.zeros((Lt, Lz, Ly, Lx, 4, 3), dtype=np.complex128)
            v[0, 0, 0, 0, s, c] = 1.0
            out.append(v)
    return out
