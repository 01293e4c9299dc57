"""Writes the stored expected values under tests/golden/ by calling only oracle/.

The paper prints no worked numeric example (no H/S values, no plane-wave
counts), so every value here comes from the oracle on the seeded inputs:
  gcounts.txt   number of plane waves |k+G| <= K_max per workload and k-point
  c1_hs.txt     sampled elements of H and S for the 2-atom workload
Run: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
from paper_1712_07206_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    with open(os.path.join(HERE, "gcounts.txt"), "w") as f:
        f.write("# config kpoint kmax n_g   (oracle plane-wave set, Sec. 2: |k+G| <= K_max)\n")
        for c in (1, 2, 3, 4, 5):
            p = inputs.CONFIGS[c]()
            for k in range(p.n_k):
                n3 = oracle.gvectors(p.lattice, p.k_frac[k], p.kmax[k])
                f.write(f"{c} {k} {p.kmax[k]:.15f} {len(n3)}\n")
    p = inputs.config1()
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    cols = [0, 1, 57, 150, len(n3) - 1]
    H, S = oracle.hs_columns(p, 0, n3, cols)
    rows = [0, 3, 99, 200, len(n3) - 1]
    with open(os.path.join(HERE, "c1_hs.txt"), "w") as f:
        f.write("# row col Re(H) Im(H) Re(S) Im(S)  (oracle, Eqs. (def_hamilton), (def_overlap))\n")
        for ci, c in enumerate(cols):
            for r in rows:
                h, s = H[ci, r], S[ci, r]
                f.write(f"{r} {c} {h.real:.17e} {h.imag:.17e} {s.real:.17e} {s.imag:.17e}\n")


if __name__ == "__main__":
    main()
