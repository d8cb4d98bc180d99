"""Polar long-range coupling g^L (Sec. 3.2) in the grid-DFT linewidths through the C ABI, against
the FP64 oracle (1e-5 relative on Gamma_nk, floor 1e-6 of the median)."""
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


def _polar(na, seed=3):
    rng = np.random.default_rng(seed)
    zs = rng.normal(size=(na, 3, 3)) * 0.5 + 2.0 * np.eye(3)[None]
    zs -= zs.mean(axis=0, keepdims=True) if na > 1 else 0.0      # acoustic sum rule where it applies
    e = rng.normal(size=(3, 3)) * 0.3
    return {"Zstar": zs, "eps_inf": 8.0 * np.eye(3) + e @ e.T, "alpha": 1.5}


@pytest.mark.parametrize("case", ["toy", "si_like"])
def test_polar_linewidths(pg, case):
    if case == "toy":
        mat, prm = W.toy(seed=0)
        ks_sel = None
    else:
        mat, prm = W.si_like(seed=0, nk=8)
        ks_sel = None
    pol = _polar(mat.na)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        ctx.set_polar(pol["Zstar"], pol["eps_inf"], pol["alpha"])
        ks, bs, gam = ctx.linewidths_rta(pg.make_params(prm, precision=7))
        ctx.set_polar(None)
        _, _, g0 = ctx.linewidths_rta(pg.make_params(prm, precision=7))
    k2, b2, ref = elph.linewidths_rta(mat, prm, k_indices=ks_sel, polar=pol)
    assert np.array_equal(ks, k2) and np.array_equal(bs, b2)
    err = rel_err(gam, ref)
    print(f"{case} polar: max rel err {err:.3e}, mean Gamma change {np.mean(gam / g0):.3f}x")
    assert err <= RTOL
    assert not np.allclose(gam, g0, rtol=1e-2)


def test_polar_argument_checks(pg):
    mat, prm = W.toy(seed=0)
    pol = _polar(1)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.set_polar(pol["Zstar"], -np.eye(3), 1.0)
        assert e.value.status == -1                   # eps_inf not positive definite
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.set_polar(pol["Zstar"], pol["eps_inf"], 0.0)
        assert e.value.status == -1                   # alpha <= 0
        ctx.set_polar(pol["Zstar"], pol["eps_inf"], pol["alpha"])
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.linewidths_rta(pg.make_params(prm, precision=0))
        assert e.value.status == -9                   # ERR_UNSUPPORTED outside the grid-DFT stage 2
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.phonon_rates_elph(pg.make_params(prm, precision=7), 3)
        assert e.value.status == -9
