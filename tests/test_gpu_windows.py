"""Windows on both states of a transition (window_final = 1, Sec. 5.2) in the grid-DFT stage 2
through the C ABI, against the FP64 oracle (1e-5 relative, floor 1e-6 of the median)."""
import numpy as np
import pytest

from oracle import elph
from workloads import synthetic as W

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def rel_err(a, b, floor_of=np.median):
    floor = 1e-6 * floor_of(np.abs(b))
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


@pytest.fixture(scope="module")
def pg():
    import paper_2111_14999_b300 as pg
    return pg


@pytest.fixture(scope="module")
def si8():
    return W.si_like(seed=0, nk=8)


def test_einstein_final_state_window(pg):
    mat, prm = W.tb_einstein(eps0=0.05, t=0.25, n=8, mu=0.1)
    prm = prm.with_(window_eV=0.43, window_final=1)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        ks, bs, gam = ctx.linewidths_rta(pg.make_params(prm, precision=7))
    k2, b2, ref = elph.linewidths_rta(mat, prm)
    assert np.array_equal(ks, k2)
    assert rel_err(gam, ref) <= RTOL


@pytest.mark.parametrize("population", [False, True])
def test_si_like_final_state_window(pg, si8, population):
    mat, prm = si8
    prm = prm.with_(window_final=1, population_delta=1e-4 if population else 0.0)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        ks, bs, gam = ctx.linewidths_rta(pg.make_params(prm, precision=7))
        wide = ctx.linewidths_rta(pg.make_params(prm.with_(window_final=0), precision=7))[2]
    k2, b2, ref = elph.linewidths_rta(mat, prm)
    assert np.array_equal(ks, k2) and np.array_equal(bs, b2)
    err = rel_err(gam, ref)
    print(f"Si-like 8^3 final-state window (population={population}): max rel err {err:.3e}")
    assert err <= RTOL
    assert np.all(gam <= wide * (1 + 1e-6)) and np.any(gam < 0.999 * wide)


def test_si_like_phonon_rates_final_state_window(pg, si8):
    mat, prm = si8
    prm = prm.with_(window_final=1)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        P = ctx.phonon_rates_elph(pg.make_params(prm, precision=7), 3 * mat.na)
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.linewidths_rta(pg.make_params(prm, precision=5))
        assert e.value.status == -9                  # ERR_UNSUPPORTED outside the grid-DFT stage 2
    ref = elph.phonon_rates_elph(mat, prm)
    assert rel_err(P, ref, np.max) <= RTOL
