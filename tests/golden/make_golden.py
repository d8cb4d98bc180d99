"""Write the stored expected values under tests/golden/ (calls only the oracle).

The paper prints no worked numerical example for this path (its timing and
linewidth plots are figures), so the stored values are oracle outputs on the
seeded toy crystal, kept to detect drift of the oracle itself.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import elph  # noqa: E402
from workloads import synthetic as W  # noqa: E402


def main():
    mat, prm = W.toy(seed=0)
    ks, bs, gam = elph.linewidths_rta(mat, prm)
    path = os.path.join(HERE, "toy_seed0_gamma.txt")
    with open(path, "w") as f:
        f.write("# Gamma_nk (eV) of the seeded toy crystal (workloads.toy(seed=0)), FP64 oracle,\n")
        f.write("# Sec. 4.2 Eq. 29 with the readings of oracle/elph.py.  columns: k_index band gamma_eV\n")
        for k, b, g in zip(ks, bs, gam):
            f.write(f"{k:d} {b:d} {g:.17e}\n")
    print("wrote", path, len(ks))


if __name__ == "__main__":
    main()
