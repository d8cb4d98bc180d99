"""Three-phonon coupling and the three-phonon diagonal of the phonon scattering matrix (Sec. 3.1,
Sec. 4.3) through the C ABI against the FP64 oracle: 1e-5 relative, floor 1e-6 of the maximum."""
import dataclasses

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


def _run(pg, mat, anh, prm):
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        ctx.set_force_constants3(anh)
        return ctx.three_phonon_rates(pg.make_params(prm), 3 * mat.na)


@pytest.mark.parametrize("offsite", [None, ((1, 0, 0), (0, 1, 0))])
def test_einstein_three_phonon(pg, offsite):
    mat, anh, prm = W.einstein3(n=6, offsite=offsite)
    A = _run(pg, mat, anh, prm)
    ref = elph.three_phonon_diag(mat, anh, prm)
    assert rel_err(A, ref) <= RTOL and np.max(A) > 0


def test_si_like_three_phonon(pg):
    mat, anh, prm = W.three_phonon_si_like(seed=0, nq=6)
    A = _run(pg, mat, anh, prm)
    ref = elph.three_phonon_diag(mat, anh, prm)
    err = rel_err(A, ref)
    print(f"Si-like 6^3 three-phonon diagonal: max rel err {err:.3e}")
    assert err <= RTOL and np.max(A) > 0


@pytest.mark.parametrize("nq", [(2, 3, 40), (5, 4, 3)])
def test_si_like_three_phonon_uneven_grids(pg, nq):
    """Grids whose z lines are longer than one block's 32 q~ (two chunks per line) or short enough
    for ten lines per block, with different residue sets per axis."""
    mat, anh, prm = W.three_phonon_si_like(seed=0, nq=6)
    prm = dataclasses.replace(prm, nk=nq, nq=nq)
    A = _run(pg, mat, anh, prm)
    ref = elph.three_phonon_diag(mat, anh, prm)
    err = rel_err(A, ref)
    print(f"Si-like {nq} three-phonon diagonal: max rel err {err:.3e}")
    assert err <= RTOL and np.max(A) > 0


def test_three_phonon_argument_checks(pg):
    mat, anh, prm = W.einstein3(n=4)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.three_phonon_rates(pg.make_params(prm), 6)
        assert e.value.status == -2                  # ERR_ORDER: no third-order constants
        ctx.set_force_constants3(anh)
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.three_phonon_rates(pg.make_params(prm), 5)
        assert e.value.status == -1                  # ERR_ARG: wrong output size
