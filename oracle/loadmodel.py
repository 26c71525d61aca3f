"""Domain count and load of Sec. IV-B (Eq. 6-7).  Test infrastructure only.

n_domain = V / (2 V_domain): domains of one colour processed in parallel.
load     = n_domain / (N_core * ceil(n_domain / N_core)).
"""
from __future__ import annotations

import math


def n_domain(local_volume: int, domain_volume: int = 8 * 4 ** 3) -> float:
    return 0.5 * local_volume / domain_volume


def load(n_dom: int, n_core: int = 60) -> float:
    return n_dom / (n_core * math.ceil(n_dom / n_core))


def load_mixed(counts, n_core: int = 60) -> float:
    """Average load over nodes that hold different domain counts (non-uniform split)."""
    busiest = max(counts)
    return sum(counts) / (len(counts) * n_core * math.ceil(busiest / n_core))
