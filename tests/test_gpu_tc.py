"""Tensor-core (tcgen05) precisions vs the FP64 oracle through the C ABI.

Tolerance for the split precisions: 1e-5 relative on Gamma_nk, measured as
max |G_gpu - G_ref| / max(|G_ref|, 1e-6 * median |G_ref|) so that states with
a vanishing linewidth are compared absolutely.
"""
import numpy as np
import pytest

from oracle import elph
from workloads import synthetic as W

pytestmark = pytest.mark.gpu

SPLIT_RTOL = 1e-5
SINGLE_RTOL = 5e-2      # single-pass BF16 / TF32 are reported, not held to 1e-5


def rel_err(a, b):
    floor = 1e-6 * np.median(np.abs(b))
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


@pytest.fixture(scope="module")
def pg():
    import paper_2111_14999_b300 as pg
    return pg


@pytest.fixture(scope="module")
def toy_ref():
    ref = np.loadtxt(__file__.replace("test_gpu_tc.py", "golden/toy_seed0_gamma.txt"))
    return ref


@pytest.fixture(scope="module")
def toy_ctx(pg):
    mat, prm = W.toy(seed=0)
    ctx = pg.PhoebeGPU(0)
    ctx.set_material(mat)
    yield ctx, prm
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(1, SPLIT_RTOL), (2, SPLIT_RTOL), (5, SPLIT_RTOL), (3, SINGLE_RTOL),
                                      (4, SINGLE_RTOL), (6, 1e-4), (7, SPLIT_RTOL)])
def test_toy_full_grid_precisions(pg, toy_ctx, toy_ref, prec, tol):
    ctx, prm = toy_ctx
    ks, bs, gam = ctx.linewidths_rta(prm, precision=prec)
    assert np.array_equal(ks, toy_ref[:, 0].astype(int)) and np.array_equal(bs, toy_ref[:, 1].astype(int))
    err = rel_err(gam, toy_ref[:, 2])
    print(f"toy precision {prec}: max rel err {err:.3e}")
    assert err <= tol


def test_toy_ragged_batches(pg, toy_ctx, toy_ref):
    ctx, prm = toy_ctx
    ks, bs, gam = ctx.linewidths_rta(prm, precision=5, max_batch_states=37)
    assert rel_err(gam, toy_ref[:, 2]) <= SPLIT_RTOL


def test_toy_subset_and_coarse_k(pg, toy_ctx):
    ctx, prm = toy_ctx
    mat, _ = W.toy(seed=0)
    p2 = prm.with_(nk=(4, 4, 4), nq=(8, 8, 8), k_subset=[0, 5, 17, 63])
    ks, bs, gam = ctx.linewidths_rta(p2, precision=5)
    k2, b2, ref = elph.linewidths_rta(mat, p2, k_indices=[0, 5, 17, 63])
    assert np.array_equal(ks, k2)
    assert rel_err(gam, ref) <= SPLIT_RTOL


@pytest.mark.parametrize("prec", [1, 5, 7])
def test_einstein_closed_form_split(pg, prec):
    mat, prm = W.tb_einstein(eps0=0.05, t=0.25, lam=0.215, n=8, mu=0.1)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        ks, bs, gam = ctx.linewidths_rta(prm, precision=prec)
    _, _, ref = elph.linewidths_rta(mat, prm)
    assert rel_err(gam, ref) <= SPLIT_RTOL


@pytest.fixture(scope="module")
def si():
    mat, prm = W.si_like(seed=0)
    tab = elph.electron_table(mat, prm)
    return mat, prm, tab


@pytest.mark.parametrize("prec", [5, 7])
def test_si_like_full_grid_sampled(pg, si, prec):
    """The benchmark configuration: every active state of the 40^3 x 40^3 Si-like grid in split
    FP16 (precision 5) or as grid DFTs (precision 7, the benchmarked mode, default batches),
    compared on a seeded sample of k points with the FP64 oracle."""
    mat, prm, tab = si
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        ks, bs, gam = ctx.linewidths_rta(prm, precision=prec)
        st = ctx.stats()
    eg = tab[1][tab[3]]
    k_all, b_all = elph.active_states(eg, prm.mu_eV, prm.window_eV)
    assert np.array_equal(ks, k_all) and np.array_equal(bs, b_all)
    assert np.all(gam >= 0)
    rng = np.random.default_rng(3)
    pick = np.sort(rng.choice(np.unique(k_all), 6, replace=False))
    k2, b2, ref = elph.linewidths_rta(mat, prm, k_indices=pick, table=tab)
    sel = np.isin(ks, pick)
    err = rel_err(gam[sel], ref)
    print(f"Si-like full grid precision {prec}: {len(gam)} states, sampled max rel err {err:.3e}, stats {st}")
    assert err <= SPLIT_RTOL


@pytest.mark.parametrize("prec", [1, 2, 7])
def test_si_like_subset_split_bf16_tf32(pg, si, prec):
    mat, prm, tab = si
    eg = tab[1][tab[3]]
    k_all, _ = elph.active_states(eg, prm.mu_eV, prm.window_eV)
    pick = np.sort(np.random.default_rng(4).choice(np.unique(k_all), 4, replace=False))
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        ks, bs, gam = ctx.linewidths_rta(prm, precision=prec, k_subset=pick)
    k2, b2, ref = elph.linewidths_rta(mat, prm, k_indices=pick, table=tab)
    assert np.array_equal(ks, k2)
    err = rel_err(gam, ref)
    print(f"Si-like subset precision {prec}: max rel err {err:.3e}")
    assert err <= SPLIT_RTOL


def test_grid_dft_matches_tensor_core_stage2_on_full_grid(pg, si):
    """Stage 2 as the separable grid DFT (FP32) against the tensor-core GEMM (split FP16) over every
    active state of the Si-like 40^3 grid: both approximate the same FP64 sum to ~2e-6."""
    mat, prm, tab = si
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        k5, b5, g5 = ctx.linewidths_rta(prm, precision=5)
        k7, b7, g7 = ctx.linewidths_rta(prm, precision=7, max_batch_states=700)   # ragged batches
    assert np.array_equal(k5, k7) and np.array_equal(b5, b7)
    assert rel_err(g7, g5) <= 2 * SPLIT_RTOL


def test_grid_dft_unpaired_and_half_grid_residues(pg):
    """R_p set without inversion symmetry and with R_x = +-Nx/2: the grid-DFT rows for a residue
    without its negative, for a residue pair whose planes hold different ry sets (y groups with
    absent combinations), for r = 0 and for r = Nx/2 (real phase factors), against the oracle."""
    import dataclasses
    mat, prm = W.toy(seed=0)
    keep = mat.Rp[:, 0] != 1                      # residue 1 (mod 8) gone, 7 keeps no partner
    # residue 4 = Nx / 2; residues 2 and 6 = -2 whose planes hold different ry residues
    extra = np.array([[4, 0, 0], [-4, 1, 0], [2, 1, 0], [-2, 0, 0]], dtype=np.int32)
    rng = np.random.default_rng(7)
    shape = (mat.g.shape[0], len(extra)) + mat.g.shape[2:]
    g_extra = 0.05 * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    Rp = np.concatenate([mat.Rp[keep], extra]).astype(np.int32)
    mat2 = dataclasses.replace(mat, Rp=Rp, wp=np.ones(len(Rp)),
                               g=np.concatenate([mat.g[:, keep], g_extra], axis=1))
    ks = [0, 5, 17, 63, 200, 511]
    p2 = prm.with_(k_subset=ks)
    k_ref, b_ref, ref = elph.linewidths_rta(mat2, p2, k_indices=ks)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat2)
        k7, b7, g7 = ctx.linewidths_rta(p2, precision=7)
        k5, b5, g5 = ctx.linewidths_rta(p2, precision=5)
    assert np.array_equal(k7, k_ref) and np.array_equal(b7, b_ref)
    assert rel_err(g5, ref) <= SPLIT_RTOL
    err = rel_err(g7, ref)
    print(f"asymmetric R_p set, grid DFT: max rel err {err:.3e}")
    assert err <= SPLIT_RTOL
