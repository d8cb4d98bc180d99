"""FP64 grid DFT (precision 8) against the FP64 oracle at 1e-10, and the FP64 paths on the
Si-like crystal against stored oracle values: 512+ seeded states and a full kx slab of the
40^3 x 40^3 workload (tests/golden/make_golden_si.py, which calls only the oracle)."""
import os

import numpy as np
import pytest

from oracle import elph
from workloads import synthetic as W

pytestmark = pytest.mark.gpu

RTOL_FP64 = 1e-10
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
PREC_FP64, PREC_FP64_DFT = 0, 8


@pytest.fixture(scope="module")
def pg():
    import paper_2111_14999_b300 as pg
    return pg


@pytest.fixture(scope="module")
def toy_ctx(pg):
    mat, prm = W.toy(seed=0)
    ctx = pg.PhoebeGPU(0)
    ctx.set_material(mat)
    yield ctx, mat, prm
    ctx.close()


@pytest.fixture(scope="module")
def si_ctx(pg):
    mat, prm = W.si_like(seed=0)
    ctx = pg.PhoebeGPU(0)
    ctx.set_material(mat)
    yield ctx, mat, prm
    ctx.close()


def _golden(name):
    ref = np.loadtxt(os.path.join(GOLDEN, name))
    return ref[:, 0].astype(int), ref[:, 1].astype(int), ref[:, 2]


def test_toy_full_grid(toy_ctx):
    ctx, mat, prm = toy_ctx
    ks, bs, gam = ctx.linewidths_rta(prm, precision=PREC_FP64_DFT)
    k2, b2, ref = _golden("toy_seed0_gamma.txt")
    assert np.array_equal(ks, k2) and np.array_equal(bs, b2)
    np.testing.assert_allclose(gam, ref, rtol=RTOL_FP64, atol=0)


def test_toy_ragged_batches_and_stats(toy_ctx):
    ctx, mat, prm = toy_ctx
    ctx.set_profiling(True)
    ks, bs, gam = ctx.linewidths_rta(prm, precision=PREC_FP64_DFT, max_batch_states=7)
    st = ctx.stats()
    ctx.set_profiling(False)
    _, _, ref = _golden("toy_seed0_gamma.txt")
    np.testing.assert_allclose(gam, ref, rtol=RTOL_FP64, atol=0)
    assert st["stage2_launches"] >= 1024 // 7
    assert 0 < st["pairs_executed"] <= 1024 * 512


@pytest.mark.parametrize("nk,nq,sub", [((4, 4, 4), (8, 8, 8), None), ((8, 8, 8), (4, 2, 8), [0, 3, 77, 200, 511])])
def test_toy_commensurate_grids(toy_ctx, nk, nq, sub):
    ctx, mat, prm = toy_ctx
    p2 = prm.with_(nk=nk, nq=nq)
    if sub is not None:
        p2 = p2.with_(k_subset=sub)
    ks, bs, gam = ctx.linewidths_rta(p2, precision=PREC_FP64_DFT)
    k2, b2, ref = elph.linewidths_rta(mat, p2, k_indices=sub)
    assert np.array_equal(ks, k2) and np.array_equal(bs, b2)
    np.testing.assert_allclose(gam, ref, rtol=RTOL_FP64)


@pytest.mark.parametrize("nw,na", [(3, 1), (5, 3), (8, 2), (12, 2)])
def test_shapes_without_fp32_kernels(pg, nw, na):
    """The FP64 grid DFT is generic in (N_w, 3 N_at): shapes the FP32 kernels are not built for."""
    rng = np.random.default_rng([29, nw, na])
    mat, prm = W.material_of_shape(f"shape64_{nw}_{na}", nw, na, 60, 6, rng, g_budget_bytes=32e6)
    sub = np.sort(np.random.default_rng([4, nw, na]).choice(6 ** 3, 10, replace=False))
    prm = prm.with_(k_subset=sub, window_eV=0.0)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        ks, bs, gam = ctx.linewidths_rta(pg.make_params(prm, precision=PREC_FP64_DFT))
    k2, b2, ref = elph.linewidths_rta(mat, prm, k_indices=sub)
    assert np.array_equal(ks, k2) and np.array_equal(bs, b2)
    assert np.max(ref) > 0
    np.testing.assert_allclose(gam, ref, rtol=RTOL_FP64)


def test_window_subset_and_empty(toy_ctx):
    ctx, mat, prm = toy_ctx
    p2 = prm.with_(window_eV=0.8, k_subset=np.arange(0, 512, 3))
    ks, bs, gam = ctx.linewidths_rta(p2, precision=PREC_FP64_DFT)
    k2, b2, ref = elph.linewidths_rta(mat, p2, k_indices=np.arange(0, 512, 3))
    assert len(ks) > 0 and np.array_equal(ks, k2) and np.array_equal(bs, b2)
    np.testing.assert_allclose(gam, ref, rtol=RTOL_FP64)
    ks, bs, gam = ctx.linewidths_rta(prm.with_(window_eV=1e-9), precision=PREC_FP64_DFT)
    assert len(ks) == 0


def test_unsupported_options_are_refused(pg, toy_ctx):
    ctx, mat, prm = toy_ctx
    with pytest.raises(pg.PhoebeGPUError):
        ctx.linewidths_rta(prm.with_(sampler=2, sample_fraction=0.1), precision=PREC_FP64_DFT)


@pytest.mark.parametrize("name", ["si_like_seed0_sample_gamma.txt", "si_like_seed0_slab13_gamma.txt"])
@pytest.mark.parametrize("prec", [PREC_FP64_DFT, PREC_FP64])
def test_si_like_against_stored_oracle(si_ctx, name, prec):
    """Both FP64 paths on the Si-like 40^3 x 40^3 workload: 512+ seeded states, and every active
    state of one kx plane, each against the oracle's stored values at 1e-10."""
    ctx, mat, prm = si_ctx
    k2, b2, ref = _golden(name)
    ks, bs, gam = ctx.linewidths_rta(prm, precision=prec, k_subset=np.unique(k2))
    assert np.array_equal(ks, k2) and np.array_equal(bs, b2)
    assert len(ref) >= 512
    np.testing.assert_allclose(gam, ref, rtol=RTOL_FP64, atol=0)
