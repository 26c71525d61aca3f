"""Partition of the lattice over ranks for the multi-GPU form of the solver (Sec. III-E, Fig. 4).

Host logic only (plain Python): this build runs on one GPU, so no library path uses it; the
partition and its exchange schedule are exercised on CPU ranks (tests/test_partition_cpu.py).

The lattice is cut into a grid of hyper-rectangles of whole Schwarz domains.  Every rank
owns N_mu / grid_mu domains in direction mu, and that count must be even: then a domain's
colour (the parity of its global domain coordinates) equals the parity of its local ones,
so each rank can run the colour sweeps of the multiplicative Schwarz method on its own
domains with the global two-colouring, and only two things cross rank boundaries:
  * before each half-sweep, the one-site-thick boundary planes of the current solution
    (in the library's form: the projected half-spinors of the face buffers) go to the
    neighbouring ranks, which need them for the residual of their boundary domains;
  * the inner products of the outer Krylov solver are all-reduced (FP64).
"""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass
class RankBlock:
    rank: int
    coords: tuple          # position in the rank grid (x, y, z, t)
    offset: tuple          # first owned site, global coordinates (x, y, z, t)
    extent: tuple          # owned sites per direction (x, y, z, t)
    neighbours: dict = field(default_factory=dict)   # (mu, +1 / -1) -> rank, partitioned mu only


def rank_of(coords, grid) -> int:
    """Rank of a grid position, x fastest."""
    r = 0
    for mu in (3, 2, 1, 0):
        r = r * grid[mu] + coords[mu]
    return r


def plan(dims, domain, grid) -> list[RankBlock]:
    """The blocks of a rank grid `grid` = (gx, gy, gz, gt) over a lattice `dims` split into
    domains `domain`.  Raises ValueError unless every rank owns an even number (>= 2) of
    whole domains in every direction."""
    dims, domain, grid = tuple(dims), tuple(domain), tuple(grid)
    for mu in range(4):
        if dims[mu] % domain[mu]:
            raise ValueError(f"domain extent {domain[mu]} does not divide {dims[mu]}")
        n = dims[mu] // domain[mu]
        if grid[mu] < 1 or n % grid[mu]:
            raise ValueError(f"{grid[mu]} ranks do not divide {n} domains in direction {mu}")
        per = n // grid[mu]
        if per < 2 or per % 2:
            raise ValueError(f"{per} domains per rank in direction {mu}: need an even number >= 2")
    extent = tuple(dims[mu] // grid[mu] for mu in range(4))
    blocks = []
    nranks = grid[0] * grid[1] * grid[2] * grid[3]
    for r in range(nranks):
        c, q = [], r
        for mu in range(4):
            c.append(q % grid[mu])
            q //= grid[mu]
        c = tuple(c)
        b = RankBlock(r, c, tuple(c[mu] * extent[mu] for mu in range(4)), extent)
        for mu in range(4):
            if grid[mu] == 1:
                continue
            for step in (+1, -1):
                nc = list(c)
                nc[mu] = (c[mu] + step) % grid[mu]
                b.neighbours[(mu, step)] = rank_of(nc, grid)
        blocks.append(b)
    return blocks


def halo_bytes_per_half_sweep(block: RankBlock, bytes_per_face_site: int = 48) -> int:
    """Bytes one rank sends per Schwarz half-sweep: the faces of the boundary domains of the
    colour just updated (half of each boundary plane) in every partitioned direction, both
    sides, 12 reals per face site (FP32 by default: the projected half-spinor, Sec. III-E)."""
    total = 0
    for (mu, _step) in block.neighbours:
        face = 1
        for nu in range(4):
            if nu != mu:
                face *= block.extent[nu]
        total += face // 2 * bytes_per_face_site
    return total
