"""Phonon-electron rates P^{el-ph}_{q nu} (Sec. 4.3) from the grid-DFT stage 2 through the C ABI,
against the FP64 oracle.  Tolerance 1e-5 relative, measured against max(|P_ref|, 1e-6 max |P_ref|)
so that modes with a vanishing rate are compared absolutely."""
import numpy as np
import pytest

from oracle import elph
from workloads import synthetic as W

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def rel_err(a, b):
    floor = 1e-6 * np.max(np.abs(b))
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


@pytest.fixture(scope="module")
def pg():
    import paper_2111_14999_b300 as pg
    return pg


def _rates(pg, mat, prm):
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        return ctx.phonon_rates_elph(pg.make_params(prm, precision=7), 3 * mat.na)


def test_toy_phonon_rates(pg):
    mat, prm = W.toy(seed=0)
    P = _rates(pg, mat, prm)
    ref = elph.phonon_rates_elph(mat, prm)
    err = rel_err(P, ref)
    print(f"toy phonon rates: max rel err {err:.3e}")
    assert P.shape == ref.shape and err <= RTOL
    assert np.all(P[0] == 0.0)                      # dead acoustic modes at Gamma


def test_einstein_phonon_rates_degenerate_modes(pg):
    mat, prm = W.tb_einstein(eps0=0.05, t=0.25, n=8, mu=0.1)
    P = _rates(pg, mat, prm)
    ref = elph.phonon_rates_elph(mat, prm)
    assert rel_err(P, ref) <= RTOL
    assert np.allclose(P[:, 0], P[:, 1], rtol=1e-12) and np.allclose(P[:, 0], P[:, 2], rtol=1e-12)


def test_si_like_phonon_rates_with_window(pg):
    mat, prm = W.si_like(seed=0, nk=8)
    P = _rates(pg, mat, prm)
    ref = elph.phonon_rates_elph(mat, prm)
    err = rel_err(P, ref)
    print(f"Si-like 8^3 phonon rates: max rel err {err:.3e}")
    assert err <= RTOL and np.max(P) > 0


def test_phonon_rates_leave_linewidths_unchanged_and_check_arguments(pg):
    mat, prm = W.toy(seed=0)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        p7 = pg.make_params(prm, precision=7)
        k1, b1, g1 = ctx.linewidths_rta(p7)
        ctx.phonon_rates_elph(p7, 3)
        k2, b2, g2 = ctx.linewidths_rta(p7)
        assert np.array_equal(k1, k2) and np.allclose(g1, g2, rtol=1e-12)
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.phonon_rates_elph(pg.make_params(prm, precision=5), 3)
        assert e.value.status == -9                  # ERR_UNSUPPORTED: not the grid-DFT stage 2
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.phonon_rates_elph(p7, 2)
        assert e.value.status == -1                  # ERR_ARG: wrong output size
