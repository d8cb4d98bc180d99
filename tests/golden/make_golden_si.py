"""Write stored oracle values for the Si-like crystal (calls only the oracle).

The FP64 oracle costs about two seconds per Si-like k point on 40^3 q, too slow to run
inside a GPU test for hundreds of states, so its values are computed once here and
stored:

* ``si_like_seed0_sample_gamma.txt``: Gamma_nk of every active state on seeded active k
  points of the Si-like 40^3 x 40^3 workload (workloads.si_like(seed=0)), at least 512
  states;
* ``si_like_seed0_slab13_gamma.txt``: Gamma_nk of every active state of the kx = 13 plane
  of the same k grid (a full k-slab).

Run from the repository root:  python tests/golden/make_golden_si.py [sample|slab]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import elph  # noqa: E402
from workloads import synthetic as W  # noqa: E402

SAMPLE_STATES = 512
SLAB_KX = 13


def sample_k(ks: np.ndarray, n_states: int, seed: int = 7) -> np.ndarray:
    """Seeded active k points, drawn until their active states number at least n_states."""
    uk = np.unique(ks)
    order = np.random.default_rng(seed).permutation(len(uk))
    counts = np.bincount(ks, minlength=uk.max() + 1)
    tot, pick = 0, []
    for i in order:
        pick.append(uk[i])
        tot += counts[uk[i]]
        if tot >= n_states:
            break
    return np.sort(np.array(pick))


def write(path, header, ks, bs, gam):
    with open(path, "w") as f:
        for line in header:
            f.write("# " + line + "\n")
        f.write("# columns: k_index band gamma_eV\n")
        for k, b, g in zip(ks, bs, gam):
            f.write(f"{k:d} {b:d} {g:.17e}\n")
    print("wrote", path, len(ks), flush=True)


def main(which):
    mat, prm = W.si_like(seed=0)
    tab = elph.electron_table(mat, prm)
    eg = tab[1][tab[3]]
    ks, _ = elph.active_states(eg, prm.mu_eV, prm.window_eV)
    common = ["Gamma_nk (eV) of the seeded Si-like crystal (workloads.si_like(seed=0)): 40^3 k x 40^3 q,",
              "T = 300 K, sigma = 0.02 eV, window +-0.5 eV; FP64 oracle, Sec. 4.2 Eq. 29 with the readings",
              "of oracle/elph.py (Gamma averaged over degenerate active bands)."]
    if which in ("sample", "all"):
        pick = sample_k(ks, SAMPLE_STATES)
        t0 = time.time()
        k2, b2, g = elph.linewidths_rta(mat, prm, k_indices=pick, table=tab)
        write(os.path.join(HERE, "si_like_seed0_sample_gamma.txt"),
              common + [f"Every active state on {len(pick)} seeded active k points (numpy default_rng(7) "
                        f"permutation of the active k, drawn until >= {SAMPLE_STATES} states); "
                        f"oracle time {time.time() - t0:.0f} s."], k2, b2, g)
    if which in ("slab", "all"):
        n1, n2 = prm.nk[1], prm.nk[2]
        plane = np.unique(ks[ks // (n1 * n2) == SLAB_KX])
        t0 = time.time()
        k2, b2, g = elph.linewidths_rta(mat, prm, k_indices=plane, table=tab)
        write(os.path.join(HERE, f"si_like_seed0_slab{SLAB_KX}_gamma.txt"),
              common + [f"Every active state of the kx = {SLAB_KX} plane of the k grid ({len(plane)} active k); "
                        f"oracle time {time.time() - t0:.0f} s."], k2, b2, g)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "all")
