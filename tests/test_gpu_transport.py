"""RTA transport coefficients on the GPU (Sec. 4.2, 4.3.2) against the oracle."""
import numpy as np
import pytest

from oracle import elph
from workloads import synthetic as W

pytestmark = pytest.mark.gpu


def _close(a, b, rtol):
    return np.max(np.abs(a - b)) <= rtol * np.max(np.abs(b))


@pytest.mark.parametrize("prec,rtol", [(0, 1e-9), (5, 1e-5)])
def test_tight_binding_transport_vs_oracle(prec, rtol):
    # cubic tight-binding band with an Einstein mode: isotropic, every state scatters
    import paper_2111_14999_b300 as pg
    mat, prm = W.tb_einstein(eps0=0.05, t=0.25, n=10, mu=0.1)
    ks, bs, g = elph.linewidths_rta(mat, prm)
    want = elph.transport_rta(mat, prm, g, ks, bs)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        got = ctx.transport_rta(prm.with_(precision=prec), mat.lattice)
    for key in ("sigma", "seebeck", "kappa"):
        assert _close(got[key], want[key], rtol), key


def test_toy_fp64_conductivity_vs_oracle():
    # the toy's sums are dominated by one state with Gamma = 6.8e-7 eV (99.999 % of L_0), which makes
    # L_0 nearly rank one: S and kappa are ill-conditioned there, sigma is not
    import paper_2111_14999_b300 as pg
    mat, prm = W.toy(seed=0)
    ref = np.loadtxt(__file__.replace("test_gpu_transport.py", "golden/toy_seed0_gamma.txt"))
    ks, bs, g = ref[:, 0].astype(int), ref[:, 1].astype(int), ref[:, 2]
    want = elph.transport_rta(mat, prm, g, ks, bs)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        got = ctx.transport_rta(prm.with_(precision=0), mat.lattice)
    assert _close(got["sigma"], want["sigma"], 1e-9)


def test_si_like_split_transport_vs_oracle():
    import paper_2111_14999_b300 as pg
    mat, prm = W.si_like(seed=0, nk=6)
    ks, bs, g = elph.linewidths_rta(mat, prm)
    want = elph.transport_rta(mat, prm, g, ks, bs)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        got = ctx.transport_rta(prm.with_(precision=5), mat.lattice)
    for key in ("sigma", "seebeck", "kappa"):
        assert _close(got[key], want[key], 1e-5), key
