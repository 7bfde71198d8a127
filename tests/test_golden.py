"""Stored fixtures under tests/golden/: printed Gauss-Legendre tables (an
independent pin of the quadrature) and the oracle's config-0 energy terms
(a regression fixture written by tests/golden/make_golden.py)."""
import os

import numpy as np

import oracle as o
from paper_1307_8052_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                out.append([float(x) for x in line.split()])
    return np.array(out)


def test_gauss_legendre_matches_printed_table():
    t = _rows("gauss_legendre.txt")
    for n in sorted(set(t[:, 0].astype(int))):
        rows = t[t[:, 0] == n]
        x, w = o.gauss_legendre(n)
        for _, xi, wi in rows:
            k = int(np.argmin(np.abs(x - xi)))
            assert abs(x[k] - xi) < 1e-14 and abs(w[k] - wi) < 1e-14, (n, xi)
            # symmetric partner
            k2 = int(np.argmin(np.abs(x + xi)))
            assert abs(w[k2] - wi) < 1e-14


def test_config0_oracle_reproduces_stored_terms():
    t = _rows("config0_terms.txt")
    p = syn.config0()
    om, W = o.frequency_grid(p.nw)
    assert np.allclose(om, t[:, 1], rtol=1e-15, atol=0) and np.allclose(W, t[:, 2], rtol=1e-15, atol=0)
    E, terms = o.energy(p, om, W)
    assert np.max(np.abs(terms[0] - t[:, 3])) <= 1e-12 * np.max(np.abs(t[:, 3]))
