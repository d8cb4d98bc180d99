"""Pins of the RTA transport oracle (Sec. 4.2 fluxes and Onsager coefficients, Sec. 4.3.2), CPU only."""
import numpy as np
import pytest

from oracle import elph
from workloads import synthetic as W

HBAR = 1.054571817e-34
EV = 1.602176634e-19


def _tb(mu, n=12, t=0.25, eps0=0.05, T=300.0):
    mat, prm = W.tb_einstein(eps0=eps0, t=t, n=n, mu=mu, T_K=T)
    tab = elph.electron_table(mat, prm)
    ks, bs = elph.active_states(tab[1][tab[3]], prm.mu_eV, prm.window_eV)
    return mat, prm, tab, ks, bs


def test_constant_lifetime_conductivity_closed_form():
    # one cubic tight-binding band, constant Gamma: sigma_xx = e^2 tau/(N V) sum v_x^2 (-df/de) with
    # hbar v_x = d eps/d k_x = 2 t a sin(2 pi k_x) from eps = eps0 - 2t sum cos(k_a a), k_a = 2 pi k_frac/a (a = 1 A)
    mat, prm, tab, ks, bs = _tb(mu=0.1)
    G = 0.013
    r = elph.transport_rta(mat, prm, np.full(len(ks), G), ks, bs, table=tab)
    n = prm.nk[0]
    k = np.indices((n, n, n)).reshape(3, -1).T / n
    eps = 0.05 - 2 * 0.25 * np.sum(np.cos(2 * np.pi * k), axis=1)
    v = 2 * 0.25 * 1e-10 * EV * np.sin(2 * np.pi * k) / HBAR                        # m/s
    kT = 1.380649e-23 * prm.T_K
    f = 1 / (np.exp((eps - prm.mu_eV) * EV / kT) + 1)
    tau = HBAR / (G * EV)
    sxx = EV ** 2 * tau / (n ** 3 * 1e-30) * np.sum(v[:, 0] ** 2 * f * (1 - f) / kT)
    assert r["sigma"][0, 0] == pytest.approx(sxx, rel=1e-9)
    # cubic symmetry: isotropic, no off-diagonal terms
    assert np.allclose(np.diag(r["sigma"]), sxx, rtol=1e-9)
    assert np.max(np.abs(r["sigma"] - np.diag(np.diag(r["sigma"])))) < 1e-9 * sxx


def test_particle_hole_symmetry_of_seebeck():
    # eps(k + 1/2) = 2 eps0 - eps(k) on an even grid: with a constant lifetime S(mu) = -S(2 eps0 - mu),
    # sigma and kappa unchanged
    a = _tb(mu=0.12)
    b = _tb(mu=2 * 0.05 - 0.12)
    ra = elph.transport_rta(a[0], a[1], np.full(len(a[3]), 0.01), a[3], a[4], table=a[2])
    rb = elph.transport_rta(b[0], b[1], np.full(len(b[3]), 0.01), b[3], b[4], table=b[2])
    assert np.allclose(ra["seebeck"], -rb["seebeck"], rtol=1e-8, atol=1e-12 * np.max(np.abs(ra["seebeck"])))
    assert np.allclose(ra["sigma"], rb["sigma"], rtol=1e-8, atol=1e-12 * np.max(np.abs(ra["sigma"])))
    assert np.allclose(ra["kappa"], rb["kappa"], rtol=1e-8, atol=1e-12 * np.max(np.abs(ra["kappa"])))
    assert abs(ra["seebeck"][0, 0]) > 1e-6


def test_group_velocities_match_band_slopes():
    # Cartesian hbar v = lattice^T (1/2 pi) d eps/d k_frac, checked by central differences
    mat, _ = W.si_like(seed=0, nk=4)
    k = np.random.default_rng(3).uniform(0, 1, (6, 3))
    _, U = elph.electron_bands(k, mat)
    v = elph.group_velocities(k, mat, U)
    h = 1e-6
    d = np.zeros((6, mat.nw, 3))
    for i in range(3):
        dk = np.zeros(3)
        dk[i] = h
        ep, _ = elph.electron_bands(k + dk, mat)
        em, _ = elph.electron_bands(k - dk, mat)
        d[:, :, i] = (ep - em) / (2 * h) / (2 * np.pi)
    want = np.einsum("kbi,ia->kba", d, mat.lattice)
    assert np.allclose(v, want, rtol=1e-5, atol=1e-7 * np.max(np.abs(want)))
