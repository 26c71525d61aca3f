"""Pin the oracle's load model (Eq. 6-7) to the values the paper prints."""
import os

import numpy as np

from oracle import loadmodel as L

GOLD = os.path.join(os.path.dirname(__file__), "golden", "load_model_table3.txt")


def rows():
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            yield line.split()


def test_table3_domain_counts_and_loads():
    n = 0
    for kind, lat, nodes, ndom, pct in rows():
        if kind == "table":
            V = int(np.prod([int(v) for v in lat.split("x")]))
            nd = L.n_domain(V / int(nodes))
            assert nd == int(ndom)
            assert round(100 * L.load(int(nd))) == int(pct)
            n += 1
        elif kind == "text":
            assert round(100 * L.load(int(ndom))) == int(pct)
        elif kind == "mixed":
            counts = [int(c) for c in lat.split(",")]
            assert round(100 * L.load_mixed(counts)) == int(pct)
    assert n == 9
