"""FP64 GPU path vs the FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest

from oracle import elph
from workloads import synthetic as W

pytestmark = pytest.mark.gpu

RTOL_FP64 = 1e-10


@pytest.fixture(scope="module")
def pg():
    import paper_2111_14999_b300 as pg
    return pg


@pytest.fixture(scope="module")
def toy():
    return W.toy(seed=0)


@pytest.fixture(scope="module")
def toy_ctx(pg, toy):
    ctx = pg.PhoebeGPU(0)
    ctx.set_material(toy[0])
    yield ctx
    ctx.close()


def _degenerate_sums(g2, eps_k, eps_kq, omega, tol=1e-7):
    """Sum |g|^2 over degenerate subspaces of m' (at k+q), n (at k) and nu (at q): gauge invariant."""
    P, nw, _, nm = g2.shape
    out = np.empty_like(g2)
    for p in range(P):
        Gm = np.array([[np.abs(eps_kq[p] - eps_kq[p, i]) < tol for i in range(nw)]], dtype=float)[0]
        Gn = np.array([[np.abs(eps_k[p] - eps_k[p, i]) < tol for i in range(nw)]], dtype=float)[0]
        Gv = np.array([[np.abs(omega[p] - omega[p, i]) < tol for i in range(nm)]], dtype=float)[0]
        out[p] = np.einsum("am,bn,cv,mnv->abc", Gm, Gn, Gv, g2[p])
    return out


def test_toy_linewidths_full_grid(pg, toy, toy_ctx):
    mat, prm = toy
    ks, bs, gam = toy_ctx.linewidths_rta(prm)
    ref = np.loadtxt(__file__.replace("test_gpu_fp64.py", "golden/toy_seed0_gamma.txt"))
    assert np.array_equal(ks, ref[:, 0].astype(int)) and np.array_equal(bs, ref[:, 1].astype(int))
    np.testing.assert_allclose(gam, ref[:, 2], rtol=RTOL_FP64, atol=0)


def test_toy_ragged_batches_and_stats(pg, toy, toy_ctx):
    mat, prm = toy
    toy_ctx.set_profiling(True)
    ks, bs, gam = toy_ctx.linewidths_rta(prm, max_batch_states=7)
    st = toy_ctx.stats()
    toy_ctx.set_profiling(False)
    ref = np.loadtxt(__file__.replace("test_gpu_fp64.py", "golden/toy_seed0_gamma.txt"))
    np.testing.assert_allclose(gam, ref[:, 2], rtol=RTOL_FP64, atol=0)
    assert st["n_states"] == 1024 and st["n_q"] == 512 and st["pairs_executed"] == 1024 * 512
    assert st["kernel_launches"] > 0 and st["stage2_launches"] >= 1024 // 8
    assert st["total_ms"] > 0


def test_toy_k_grid_coarser_than_q_grid(pg, toy, toy_ctx):
    mat, prm = toy
    p2 = prm.with_(nk=(4, 4, 4), nq=(8, 8, 8))
    ks, bs, gam = toy_ctx.linewidths_rta(p2)
    k2, b2, g2 = elph.linewidths_rta(mat, p2)
    assert np.array_equal(ks, k2) and np.array_equal(bs, b2)
    np.testing.assert_allclose(gam, g2, rtol=RTOL_FP64)
    p3 = prm.with_(nk=(8, 8, 8), nq=(4, 2, 8), k_subset=[0, 3, 77, 200, 511])
    ks, bs, gam = toy_ctx.linewidths_rta(p3)
    k3, b3, g3 = elph.linewidths_rta(mat, p3, k_indices=[0, 3, 77, 200, 511])
    assert np.array_equal(ks, k3)
    np.testing.assert_allclose(gam, g3, rtol=RTOL_FP64)


def test_toy_window_subset_and_empty(pg, toy, toy_ctx):
    mat, prm = toy
    p2 = prm.with_(window_eV=0.8, k_subset=np.arange(0, 512, 3))
    ks, bs, gam = toy_ctx.linewidths_rta(p2)
    k2, b2, g2 = elph.linewidths_rta(mat, p2, k_indices=np.arange(0, 512, 3))
    assert len(ks) > 0 and np.array_equal(ks, k2) and np.array_equal(bs, b2)
    np.testing.assert_allclose(gam, g2, rtol=RTOL_FP64)
    ks, bs, gam = toy_ctx.linewidths_rta(prm.with_(window_eV=1e-9))
    assert len(ks) == 0


def test_pairs_gauge_invariant_couplings(pg, toy, toy_ctx):
    mat, _ = toy
    rng = np.random.default_rng(11)
    k = rng.uniform(-1, 1, (40, 3))
    q = rng.uniform(-1, 1, (40, 3))
    q[0] = 0.0                       # acoustic zeros: dead modes
    q[1] = [0.25, 0.25, 0.5]         # degenerate phonons
    g2, ek, ekq, om = toy_ctx.interpolate_couplings(k, q)
    r2, rk, rkq, rom = elph.couplings_for_pairs(k, q, mat)
    np.testing.assert_allclose(ek, rk, atol=1e-12)
    np.testing.assert_allclose(ekq, rkq, atol=1e-12)
    np.testing.assert_allclose(om, rom, atol=1e-9)
    a = _degenerate_sums(g2, ek, ekq, om)
    b = _degenerate_sums(r2, rk, rkq, rom)
    scale = np.max(np.abs(b))
    np.testing.assert_allclose(a, b, rtol=RTOL_FP64, atol=1e-12 * scale)


def test_einstein_closed_form_on_gpu(pg):
    mat, prm = W.tb_einstein(eps0=0.05, t=0.25, lam=0.215, n=8, mu=0.1)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        ks, bs, gam = ctx.linewidths_rta(prm)
    _, _, ref = elph.linewidths_rta(mat, prm)
    np.testing.assert_allclose(gam, ref, rtol=RTOL_FP64)


def test_degenerate_bands_averaged(pg):
    base, prm = W.tb_einstein(eps0=0.05, t=0.25, n=4, mu=0.1)
    rng = np.random.default_rng(8)
    H = np.zeros((len(base.R_H), 2, 2), dtype=np.complex128)
    H[:, 0, 0] = base.H[:, 0, 0]
    H[:, 1, 1] = base.H[:, 0, 0]
    g = (rng.normal(size=(1, 1, 2, 2, 3)) + 1j * rng.normal(size=(1, 1, 2, 2, 3))) * 0.2
    mat = W.Material("deg", 2, 1, base.mass_amu, base.lattice, base.positions, base.R_H, base.w_H, H,
                     base.R_fc, base.w_fc, base.Phi, base.Re, base.we, base.Rp, base.wp, g)
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        ks, bs, gam = ctx.linewidths_rta(prm)
    k2, b2, ref = elph.linewidths_rta(mat, prm)
    assert np.array_equal(ks, k2)
    np.testing.assert_allclose(gam, ref, rtol=RTOL_FP64)


def test_errors_are_status_codes(pg, toy):
    mat, prm = toy
    with pg.PhoebeGPU(0) as ctx:
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.linewidths_rta(prm)
        assert e.value.status == -2                      # ERR_ORDER: no inputs yet
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.set_elph_wannier(mat.Re, mat.we, mat.Rp, mat.wp, mat.g)
        assert e.value.status == -2
        bad = mat.H.copy()
        bad[0] += 0.1j
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.set_hamiltonian(mat.nw, mat.R_H, mat.w_H, bad)
        assert e.value.status == -1 and "dagger" in e.value.message
        ctx.set_material(mat)
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.linewidths_rta(prm.with_(nk=(8, 8, 8), nq=(6, 8, 8)))
        assert e.value.status == -4                      # ERR_GRID
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.linewidths_rta(prm.with_(sigma_eV=0.0))
        assert e.value.status == -1
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.linewidths_rta(prm.with_(k_subset=[5, 3]))
        assert e.value.status == -4
        s = pg.make_params(prm)
        import ctypes
        n = ctypes.c_int(10)
        out = np.empty(10)
        st = pg.lib.phoebe_gpu_linewidths_rta(ctx._ctx, ctypes.byref(s), ctypes.byref(n), None, None,
                                              out.ctypes.data_as(ctypes.c_void_p))
        assert st == -1                                  # capacity below the 1024 states
        ctx.set_memory_cap(1 << 20)
        with pytest.raises(pg.PhoebeGPUError) as e:
            ctx.linewidths_rta(prm)
        assert e.value.status == -5                      # ERR_NOMEM under the cap
        ctx.set_memory_cap(0)
        ks, bs, gam = ctx.linewidths_rta(prm.with_(k_subset=[0]))
        assert len(ks) == 2                              # context still usable


@pytest.fixture(scope="module")
def si():
    return W.si_like(seed=0)


def test_si_like_fp64_sampled_k(pg, si):
    mat, prm = si
    tab = elph.electron_table(mat, prm)
    eg = tab[1][tab[3]]
    ks_all, _ = elph.active_states(eg, prm.mu_eV, prm.window_eV)
    uk = np.unique(ks_all)
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(uk, 6, replace=False))
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        ks, bs, gam = ctx.linewidths_rta(prm.with_(k_subset=pick))
    k2, b2, ref = elph.linewidths_rta(mat, prm, k_indices=pick, table=tab)
    assert np.array_equal(ks, k2) and np.array_equal(bs, b2)
    np.testing.assert_allclose(gam, ref, rtol=RTOL_FP64)


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (5, 1e-5)])
def test_population_window_vs_oracle(prec, tol):
    import paper_2111_14999_b300 as pg
    mat, prm = W.si_like(seed=0, nk=8)
    prm = prm.with_(population_delta=1e-4)
    tab = elph.electron_table(mat, prm)
    k_all, _ = elph.active_states(tab[1][tab[3]], prm.mu_eV, 0.0, prm.T_K, prm.population_delta)
    assert 0 < len(k_all) < 512 * 8
    pick = np.unique(k_all)[::max(1, len(np.unique(k_all)) // 6)][:6]
    prm = prm.with_(k_subset=pick)
    ks, bs, ref = elph.linewidths_rta(mat, prm, k_indices=pick, table=tab)
    assert len(ks) > 0
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        k2, b2, g = ctx.linewidths_rta(prm, precision=prec)
    assert np.array_equal(k2, ks) and np.array_equal(b2, bs)
    assert np.max(np.abs(g - ref) / np.maximum(np.abs(ref), 1e-6 * np.median(np.abs(ref)))) <= tol
