"""Every (N_w, 3 N_at) shape of the grid-DFT stage 2 against the FP64 oracle on small seeded
materials of that shape (fcc cells, decaying H and g, 6^3 grids, a subset of k)."""
import numpy as np
import pytest

from oracle import elph
from workloads import synthetic as W

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def rel_err(a, b):
    floor = 1e-6 * np.median(np.abs(b))
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


@pytest.fixture(scope="module")
def pg():
    import paper_2111_14999_b300 as pg
    return pg


@pytest.mark.parametrize("nw,na", [(1, 1), (1, 2), (2, 1), (2, 2), (4, 1), (4, 2), (8, 1), (8, 2)])
def test_grid_dft_shape(pg, nw, na):
    rng = np.random.default_rng([17, nw, na])
    mat, prm = W.material_of_shape(f"shape_{nw}_{na}", nw, na, 60, 6, rng, g_budget_bytes=32e6)
    ks_all = np.arange(6 ** 3)
    sub = np.sort(np.random.default_rng([3, nw, na]).choice(ks_all, 12, replace=False))
    prm = prm.with_(k_subset=sub, window_eV=0.0)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        ks, bs, gam = ctx.linewidths_rta(pg.make_params(prm, precision=7))
    k2, b2, ref = elph.linewidths_rta(mat, prm, k_indices=sub)
    assert np.array_equal(ks, k2) and np.array_equal(bs, b2)
    err = rel_err(gam, ref)
    print(f"grid DFT shape ({nw}, {3 * na}): max rel err {err:.3e}")
    assert err <= RTOL and np.max(gam) > 0
