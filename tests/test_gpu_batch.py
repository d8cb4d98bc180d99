"""Many materials in one call (one CUDA graph for every material's stage 2) vs one call per material.

The batch runs every shape through the stage 2 that writes G to HBM and autotunes its tiles;
the per-material calls use the fused epilogue where one exists.  Both are split-precision
approximations of the same FP64 sums, so they agree to the split tolerance, and a sample is
checked against the oracle.
"""
import numpy as np
import pytest

from oracle import elph
from workloads import synthetic as W

pytestmark = pytest.mark.gpu

SPLIT_RTOL = 1e-5


def rel_err(a, b):
    floor = 1e-6 * np.median(np.abs(b))
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


SHAPES = [(4, 2, 100, 8), (5, 1, 130, 6), (8, 2, 150, 8), (3, 3, 100, 6), (13, 1, 90, 5)]


@pytest.fixture(scope="module")
def batch():
    import paper_2111_14999_b300 as pg
    mats = [W.material_of_shape(f"b{i}", nw, na, nr, n, np.random.default_rng([11, i]), g_budget_bytes=3e6)
            for i, (nw, na, nr, n) in enumerate(SHAPES)]
    ctxs = []
    for mat, _ in mats:
        c = pg.PhoebeGPU(0)
        c.set_material(mat)
        ctxs.append(c)
    yield pg, mats, ctxs
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("prec", [5, 1])
def test_batch_matches_per_material_calls(batch, prec):
    pg, mats, ctxs = batch
    jobs = [(c, pg.make_params(prm, precision=prec)) for c, (_, prm) in zip(ctxs, mats)]
    res, info = pg.binding.linewidths_rta_batch(jobs)
    assert info["graph_nodes"] >= 2 * len(mats) and info["recorded_launches"] >= len(mats)
    for (tn, tk) in info["tiles"]:
        assert tn in (128, 256) and tk in (1, 2, 4)
    for (c, (mat, prm)), (k, b, g) in zip(zip(ctxs, mats), res):
        k1, b1, g1 = c.linewidths_rta(prm, precision=prec)
        assert np.array_equal(k, k1) and np.array_equal(b, b1)
        assert len(g) > 0
        assert rel_err(g, g1) <= 2 * SPLIT_RTOL


def test_batch_fixed_tiles_and_oracle_sample(batch):
    pg, mats, ctxs = batch
    jobs = [(c, pg.make_params(prm, precision=5)) for c, (_, prm) in zip(ctxs, mats)]
    res, info = pg.binding.linewidths_rta_batch(jobs, autotune=0, n_streams=2, g_chunk_bytes=1 << 20)
    assert all(t == (256, 2) for t in info["tiles"])
    for i in (0, 3):
        mat, prm = mats[i]
        k, b, g = res[i]
        pick = np.unique(k)[:4]
        k2, b2, ref = elph.linewidths_rta(mat, prm, k_indices=pick)
        sel = np.isin(k, pick)
        assert np.array_equal(k[sel], k2) and np.array_equal(b[sel], b2)
        assert rel_err(g[sel], ref) <= SPLIT_RTOL


def test_batch_rejects_fp64_and_reports_counts(batch):
    pg, mats, ctxs = batch
    jobs = [(c, pg.make_params(prm, precision=0)) for c, (_, prm) in zip(ctxs, mats)]
    with pytest.raises(pg.PhoebeGPUError) as e:
        pg.binding.linewidths_rta_batch(jobs)
    assert e.value.status == -9


def test_concurrent_planning_matches_one_thread(batch):
    # phase 1 on several host threads (materials overlapping on the GPU) gives the results of
    # planning one material after the other, to FP64 rounding of the atomic accumulation order
    pg, mats, ctxs = batch
    jobs = [(c, pg.make_params(prm, precision=5)) for c, (_, prm) in zip(ctxs, mats)]
    r1, i1 = pg.binding.linewidths_rta_batch(jobs, autotune=0, plan_threads=1)
    r8, i8 = pg.binding.linewidths_rta_batch(jobs, autotune=0, plan_threads=8)
    assert i1["plan_threads"] == 1 and i8["plan_threads"] == 8
    for (k1, b1, g1), (k8, b8, g8) in zip(r1, r8):
        assert np.array_equal(k1, k8) and np.array_equal(b1, b8)
        np.testing.assert_allclose(g8, g1, rtol=1e-12, atol=0)


def test_batch_rejects_a_shared_context(batch):
    pg, mats, ctxs = batch
    jobs = [(ctxs[0], pg.make_params(mats[0][1], precision=5))] * 2
    with pytest.raises(pg.PhoebeGPUError) as e:
        pg.binding.linewidths_rta_batch(jobs, capacities=[10, 10])
    assert e.value.status == -1


def test_repeated_batch_call_updates_the_kept_graph(batch):
    """A second identical batch call reuses the tile choices and updates the executable graph kept
    on the first item's context; its linewidths equal the first call's up to the order of the FP64
    atomic adds."""
    pg, mats, ctxs = batch
    jobs = [(c, pg.make_params(prm, precision=1)) for c, (_, prm) in zip(ctxs, mats)]
    res0, info0 = pg.binding.linewidths_rta_batch(jobs)
    res1, info1 = pg.binding.linewidths_rta_batch(jobs)
    assert info1["graph_reused"] == 1
    assert info1["graph_nodes"] == info0["graph_nodes"] and info1["tiles"] == info0["tiles"]
    for (k0, b0, g0), (k1, b1, g1) in zip(res0, res1):
        assert np.array_equal(k0, k1) and np.array_equal(b0, b1)
        assert rel_err(g1, g0) <= 1e-12
