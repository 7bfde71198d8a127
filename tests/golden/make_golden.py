"""Writes tests/golden/config0_terms.txt from the CPU oracle alone.

Config 0 (10 bohr cubic box, 16^3 grid, q = (0.1, 0, 0) 2 pi / a, 4 occupied +
60 empty bands, NG = 139, 8 frequencies, no PAW): the frequency terms e(w_j)
of Eqs. 1-2 and E_c for w_q = 1.  Run: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as o  # noqa: E402
from paper_1307_8052_gb300 import synthetic as syn  # noqa: E402


def main():
    p = syn.config0()
    om, W = o.frequency_grid(p.nw)
    E, terms = o.energy(p, om, W)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config0_terms.txt")
    with open(path, "w") as f:
        f.write("# Config 0 frequency terms e(w_j) and E_c (w_q = 1) from oracle/rpa_oracle.py,\n")
        f.write("# written by tests/golden/make_golden.py.  Columns: j, omega_j, W_j, e(omega_j).\n")
        for j in range(p.nw):
            f.write(f"{j} {om[j]:.17e} {W[j]:.17e} {terms[0, j]:.17e}\n")
        f.write(f"# E_c {E:.17e}\n")
    print(path)


if __name__ == "__main__":
    main()
