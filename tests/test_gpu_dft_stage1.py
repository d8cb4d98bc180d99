"""Separable stage 1 of the grid-DFT mode (precision 7) against the FP64 oracle through the C ABI.

On grid k the R_e sum of Eq. 71 is evaluated per axis over the residues R_e mod N_k (rx sum per
kx plane, ry sum, rz sum by groups {r, -r}, the k at +-kz sharing their cos and sin sums).  These
cases reach the parts the Si-like workload does not: a k grid coarser than the q grid, an odd k
grid, R_e sets whose z residues lack a partner or equal their own negative, several R_e on one
residue, and batches that cut the states of a kx plane.
"""
import dataclasses

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


def _run(pg, mat, prm, ks, **kw):
    p = prm.with_(k_subset=ks)
    k_ref, b_ref, ref = elph.linewidths_rta(mat, p, k_indices=ks)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        k7, b7, g7 = ctx.linewidths_rta(p, precision=7, **kw)
    assert np.array_equal(k7, k_ref) and np.array_equal(b7, b_ref)
    return rel_err(g7, ref)


def test_coarse_k_grid(pg):
    """k on 4^3 under q on 8^3: the stage-1 phases on the coarse grid, k+q on the fine grid."""
    mat, prm = W.toy(seed=0)
    err = _run(pg, mat, prm.with_(nk=(4, 4, 4), nq=(8, 8, 8)), [0, 5, 17, 22, 42, 63])
    print(f"coarse k, grid DFT: max rel err {err:.3e}")
    assert err <= RTOL


def test_long_z_q_grid(pg):
    """q grid 4 x 4 x 72 (more than 64 points along z) under k on 2 x 2 x 8: the fused kernel's grid
    holds one block column per jz, the z sum covers jz and 72 - jz together."""
    mat, prm = W.toy(seed=2)
    err = _run(pg, mat, prm.with_(nk=(2, 2, 8), nq=(4, 4, 72)), [0, 3, 9, 17, 26, 31])
    print(f"long z q grid, grid DFT: max rel err {err:.3e}")
    assert err <= RTOL


def test_odd_k_grid(pg):
    """5^3 grids: no residue equals its own negative except 0."""
    mat, prm = W.toy(seed=1)
    err = _run(pg, mat, prm.with_(nk=(5, 5, 5), nq=(5, 5, 5)), [0, 7, 31, 62, 124])
    print(f"odd grid, grid DFT: max rel err {err:.3e}")
    assert err <= RTOL


def test_asymmetric_re_set(pg):
    """R_e without inversion symmetry: z residue 1 (mod 8) removed so 7 keeps no partner, entries
    at R_z = +-4 (the residue N/2, its own negative), R_e = (2, 1, 2) without its negative, and
    R_e = (0, 0, 8) on the residue of (0, 0, 0)."""
    mat, prm = W.toy(seed=0)
    keep = mat.Re[:, 2] != 1
    extra = np.array([[0, 0, 4], [1, 0, -4], [2, 1, 2], [0, 0, 8]], dtype=np.int32)
    rng = np.random.default_rng(5)
    shape = (len(extra),) + mat.g.shape[1:]
    g_extra = 0.05 * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    Re = np.concatenate([mat.Re[keep], extra]).astype(np.int32)
    we = np.concatenate([mat.we[keep], np.array([1.0, 0.5, 1.0, 0.25])])
    mat2 = dataclasses.replace(mat, Re=Re, we=we, g=np.concatenate([mat.g[keep], g_extra], axis=0))
    err = _run(pg, mat2, prm, [0, 3, 64, 65, 200, 300, 448, 511])
    print(f"asymmetric R_e set, grid DFT: max rel err {err:.3e}")
    assert err <= RTOL


def test_batches_cut_a_plane(pg):
    """Batches smaller than one kx plane's states: the plane is split across batches (the
    separable stage 1 then runs per batch on the plane's part)."""
    mat, prm = W.toy(seed=0)
    ks = list(range(0, 128, 3))  # two kx planes of the 8^3 grid
    err = _run(pg, mat, prm, ks, max_batch_states=9)
    print(f"plane split across batches, grid DFT: max rel err {err:.3e}")
    assert err <= RTOL
