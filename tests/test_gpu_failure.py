"""Bounded device waits give up with a status and leave the context usable (no GPU fault).

A host-controlled 'never publish' flag: the consumer of an mbarrier phase waits for a
producer that never arrives; the wait runs out after a short limit and the call reports
PHOEBE_GPU_ERR_TIMEOUT.  Afterwards the same context runs a linewidth call normally.
"""
import time

import numpy as np
import pytest

from workloads import synthetic as W

pytestmark = pytest.mark.gpu


def test_unpublished_wait_times_out_and_context_survives():
    import paper_2111_14999_b300 as pg
    with pg.PhoebeGPU(0) as ctx:
        assert pg.lib.phoebe_gpu_selftest_wait(ctx._ctx, 1, 200000) == 0
        t0 = time.time()
        st = pg.lib.phoebe_gpu_selftest_wait(ctx._ctx, 0, 50000)   # 50 ms limit
        el = time.time() - t0
        assert st == -7
        assert "ran out" in pg.lib.phoebe_gpu_last_error(ctx._ctx).decode()
        assert 0.04 < el < 5.0
        # the context is still usable
        mat, prm = W.toy(seed=0)
        ctx.set_material(mat)
        ks, bs, g = ctx.linewidths_rta(prm, precision=5, k_subset=[3, 100])
        assert len(g) == 4 and np.all(g >= 0)
        assert pg.lib.phoebe_gpu_selftest_wait(ctx._ctx, 1, 200000) == 0
