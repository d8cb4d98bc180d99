"""Adaptive Gaussian smearing (Sec. 4.7) in the grid-DFT stage 2 through the C ABI, against the
FP64 oracle.  Tolerance 1e-5 relative on Gamma_nk (floor 1e-6 of the median)."""
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


def _gamma(pg, mat, prm):
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        return ctx.linewidths_rta(pg.make_params(prm, precision=7))


@pytest.mark.parametrize("case", ["einstein", "toy"])
def test_adaptive_smearing_small(pg, case):
    if case == "einstein":
        mat, prm = W.tb_einstein(eps0=0.05, t=0.25, n=8, mu=0.1, hop_phase=0.3)
    else:
        mat, prm = W.toy(seed=0)
    prm = prm.with_(smearing=1, sigma_min_eV=2e-3)
    ks, bs, gam = _gamma(pg, mat, prm)
    k2, b2, ref = elph.linewidths_rta(mat, prm)
    assert np.array_equal(ks, k2) and np.array_equal(bs, b2)
    err = rel_err(gam, ref)
    print(f"{case} adaptive smearing: max rel err {err:.3e}")
    assert err <= RTOL


def test_adaptive_smearing_si_like(pg):
    mat, prm = W.si_like(seed=0, nk=8)
    prm = prm.with_(smearing=1, sigma_min_eV=1e-3)
    ks, bs, gam = _gamma(pg, mat, prm)
    k2, b2, ref = elph.linewidths_rta(mat, prm)
    assert np.array_equal(ks, k2)
    err = rel_err(gam, ref)
    print(f"Si-like 8^3 adaptive smearing: max rel err {err:.3e}")
    assert err <= RTOL
    fixed = _gamma(pg, mat, prm.with_(smearing=0))[2]
    assert not np.allclose(gam, fixed, rtol=1e-2)


def test_adaptive_smearing_argument_checks(pg):
    mat, prm = W.toy(seed=0)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_hamiltonian(mat.nw, mat.R_H, mat.w_H, mat.H)
        ctx.set_force_constants(mat.na, mat.mass_amu, mat.R_fc, mat.w_fc, mat.Phi)
        ctx.set_elph_wannier(mat.Re, mat.we, mat.Rp, mat.wp, mat.g)
        ctx.nw, ctx.na = mat.nw, mat.na
        p7 = pg.make_params(prm.with_(smearing=1), precision=7)
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.linewidths_rta(p7)
        assert e.value.status == -2                  # ERR_ORDER: no lattice
        ctx.set_lattice(mat.lattice)
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.linewidths_rta(pg.make_params(prm.with_(smearing=1), precision=5))
        assert e.value.status == -9                  # ERR_UNSUPPORTED: not the grid-DFT stage 2
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.set_lattice(np.zeros((3, 3)))
        assert e.value.status == -1
        ks, bs, gam = ctx.linewidths_rta(p7)
        assert len(gam) == len(ks) and np.all(gam >= 0)
