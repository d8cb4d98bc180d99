"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics (CPU only).

Each test checks the oracle against something other than itself: a closed
form, an invariant, an exact special case, an independent library routine or
a brute-force sum.  Comments name the passage of the paper each fact follows.
"""
import numpy as np
import pytest

from oracle import elph
from workloads import synthetic as W

# independent literals for the checks below (CODATA 2018 inputs)
HBAR = 1.054571817e-34
EV = 1.602176634e-19
AMU = 1.66053906660e-27
ANG = 1e-10


@pytest.fixture(scope="module")
def toy():
    return W.toy(seed=0)


def test_unit_constants_from_codata():
    # Sec. 3.1 Eq. 4 (hbar omega from D) and Eq. 7 (zero-point length)
    assert elph.HBAR_OMEGA_EV == pytest.approx(HBAR * np.sqrt(EV / (ANG ** 2 * AMU)) / EV, rel=1e-12)
    assert elph.HBAR2_AMU_EV_A2 == pytest.approx(HBAR ** 2 / (AMU * EV * ANG ** 2), rel=1e-12)
    assert elph.KB_EV == pytest.approx(1.380649e-23 / EV, rel=1e-9)


def test_grid_order_z_fastest():
    # Sec. 5.1: points sorted by incrementing z, then y, then x
    p = elph.grid_points((2, 3, 4))
    assert np.allclose(p[1], (0, 0, 0.25)) and np.allclose(p[4], (0, 1 / 3, 0))
    assert np.allclose(p[12], (0.5, 0, 0))
    idx = elph.grid_index(p, (2, 3, 4))
    assert np.array_equal(idx, np.arange(24))
    # points outside [0,1) wrap: (1.5, -1/3, 0.75) -> (1, 2, 3)
    assert elph.grid_index(np.array([1.5, -1 / 3, 0.75]), (2, 3, 4)) == (1 * 3 + 2) * 4 + 3


def test_hamiltonian_hermitian_and_eigenpairs(toy):
    # Sec. 3.2 Eqs. 10-11: H(-R) = H(R)^dagger makes H^W_k Hermitian; U^dagger H U = diag(eps)
    mat, _ = toy
    k = np.random.default_rng(1).uniform(-1, 1, (50, 3))
    Hk = elph.wannier_hamiltonian(k, mat)
    assert np.max(np.abs(Hk - np.conj(np.swapaxes(Hk, 1, 2)))) <= 1e-14 * np.max(np.abs(Hk))
    eps, U = elph.electron_bands(k, mat)
    res = Hk @ U - U * eps[:, None, :]
    assert np.max(np.abs(res)) < 1e-13
    eye = np.conj(np.swapaxes(U, 1, 2)) @ U
    assert np.max(np.abs(eye - np.eye(mat.nw))) < 1e-13
    assert np.all(np.diff(eps, axis=1) >= 0)


def test_tight_binding_closed_form_fixes_phase_sign():
    # Eq. 10 with e^{+i k.R}: a hop -t e^{+-i phi} to +-x gives eps = eps0 - 2t sum cos(2 pi k_a + phi);
    # the opposite sign convention would give cos(2 pi k_a - phi).
    mat, _ = W.tb_einstein(eps0=0.3, t=0.4, hop_phase=0.7)
    k = np.random.default_rng(2).uniform(0, 1, (40, 3))
    eps, _ = elph.electron_bands(k, mat)
    want = 0.3 - 2 * 0.4 * np.sum(np.cos(2 * np.pi * k + 0.7), axis=1)
    assert np.allclose(eps[:, 0], want, atol=1e-13)
    wrong = 0.3 - 2 * 0.4 * np.sum(np.cos(2 * np.pi * k - 0.7), axis=1)
    assert not np.allclose(eps[:, 0], wrong, atol=1e-3)


def test_toy_phonons_closed_form(toy):
    # Eqs. 3-4: nearest-neighbour springs k=1 on simple cubic, M = 28:
    # D = diag((2k/M)(1 - cos 2 pi q_a)), hbar omega_a = c sqrt(D_aa)
    mat, _ = toy
    q = np.random.default_rng(3).uniform(0, 1, (64, 3))
    omega, z = elph.phonon_modes(q, mat)
    c = HBAR * np.sqrt(EV / (ANG ** 2 * AMU)) / EV
    want = np.sort(c * np.sqrt((2.0 / 28.0) * (1 - np.cos(2 * np.pi * q))), axis=1)
    assert np.allclose(omega, want, rtol=1e-12, atol=1e-12)


def test_acoustic_sum_rule_and_time_reversal(toy):
    # Sec. 3.1: translational invariance -> three zero modes at Gamma; Phi real -> D(-q) = conj D(q)
    mat, _ = toy
    om, _ = elph.phonon_modes(np.zeros((1, 3)), mat)
    assert np.all(np.abs(om) < 1e-6)
    q = np.random.default_rng(4).uniform(0, 1, (10, 3))
    assert np.allclose(elph.dynamical_matrix(-q, mat), np.conj(elph.dynamical_matrix(q, mat)), atol=1e-14)


def test_si_like_phonons_and_window():
    # Si-like force constants: ASR zeros at Gamma; stable spectrum (all lambda >= 0)
    pytest.importorskip("numpy")
    mat, prm = W.si_like(seed=0, nk=4)
    om, _ = elph.phonon_modes(np.zeros((1, 3)), mat)
    assert np.sum(np.abs(om) < 1e-6) == 3
    q = elph.grid_points((6, 6, 6))
    lam = np.linalg.eigvalsh(elph.dynamical_matrix(q, mat))
    assert lam.min() > -1e-10
    # NN+NNN springs: top optical mode near 76 meV
    assert 0.07 < elph.HBAR_OMEGA_EV * np.sqrt(lam.max()) < 0.08
    Hk = elph.wannier_hamiltonian(q[:20], mat)
    assert np.max(np.abs(Hk - np.conj(np.swapaxes(Hk, 1, 2)))) <= 1e-14 * np.max(np.abs(Hk))


def test_statistics_and_gaussian():
    # Sec. 4.1 Bose-Einstein, Sec. 4.2 Fermi-Dirac, Sec. 4.7 Eq. 61 Gaussian normalisation
    kT = elph.KB_EV * 300.0
    assert elph.bose_einstein(np.array([kT]), 300.0)[0] == pytest.approx(1 / (np.e - 1), rel=1e-14)
    assert elph.fermi_dirac(np.array([0.1]), 0.1, 300.0)[0] == pytest.approx(0.5)
    x = np.linspace(-1, 1, 400001)
    s = 0.05
    d = elph.gaussian_delta(x, s, 6.0)
    assert np.trapezoid(d, x) == pytest.approx(1.0, abs=1e-9)   # integrates to 1 (tail < e^-36)
    assert elph.gaussian_delta(np.array([6.0 * s + 1e-12]), s, 6.0)[0] == 0.0


def test_factorised_equals_direct_double_sum(toy):
    # Sec. 5.5 Eqs. 70-71 (R_e sum at fixed k, then R_p) re-associate Eq. 13 exactly
    mat, _ = toy
    rng = np.random.default_rng(5)
    k = rng.uniform(0, 1, (6, 3))
    q = rng.uniform(0, 1, (6, 3))
    g2_fast, *_ = elph.couplings_for_pairs(k, q, mat)
    g2_dir, *_ = elph.couplings_for_pairs(k, q, mat, direct=True)
    assert np.allclose(g2_fast, g2_dir, rtol=1e-12, atol=1e-16)


def test_direct_gamma_matches_factorised(toy):
    mat, prm = toy
    ks, bs, g_fast = elph.linewidths_rta(mat, prm, k_indices=[0, 9, 300])
    ks2, bs2, g_dir = elph.linewidths_rta(mat, prm, k_indices=[0, 9, 300], direct=True)
    assert np.array_equal(ks, ks2)
    assert np.allclose(g_fast, g_dir, rtol=1e-12)


def _coupling_from_hamiltonian(mat, c):
    """g(Re,Rp)[m][n][s a] = delta_{Rp,0} c_{s a} H(Re)[m][n] on the Hamiltonian's R set."""
    R0 = np.zeros((1, 3), dtype=np.int32)
    g = np.zeros((len(mat.R_H), 1, mat.nw, mat.nw, 3 * mat.na), dtype=np.complex128)
    g[:, 0] = mat.H[:, :, :, None] * np.asarray(c)[None, None, None, :]
    return W.Material(mat.name, mat.nw, mat.na, mat.mass_amu, mat.lattice, mat.positions,
                      mat.R_H, mat.w_H, mat.H, mat.R_fc, mat.w_fc, mat.Phi,
                      mat.R_H.copy(), mat.w_H.copy(), R0, np.ones(1), g)


def test_coupling_proportional_to_hamiltonian_fixes_daggers_and_sides(toy):
    # With g(Re,Rp) = delta_{Rp,0} c H(Re), Eq. 13 gives G^W(k,q) = c H^W_k and, by Eq. 11,
    # g_{m'n nu} = eps_nk [U_{k+q}^dagger U_k]_{m'n} (c.Z_q)_nu.  At q = 0 it is diagonal in
    # (m', n); for any q, sum_{m'} |g|^2 = eps_nk^2 |c.Z_q|^2 depends on the k side only.
    mat0, _ = toy
    c = np.array([0.7, -0.2, 0.4])
    mat = _coupling_from_hamiltonian(mat0, c)
    rng = np.random.default_rng(6)
    k = rng.uniform(0, 1, (5, 3))
    q = rng.uniform(0.05, 0.95, (5, 3))
    g2, eps_k, eps_kq, omega = elph.couplings_for_pairs(k, q, mat)
    om, z = elph.phonon_modes(q, mat)
    Zq = elph.mode_factors(om, z, mat.mass_amu, 1e-4)
    cz2 = np.abs(np.einsum("s,psv->pv", c, Zq)) ** 2                     # (p, nu)
    want = eps_k[:, :, None] ** 2 * cz2[:, None, :]                       # (p, n, nu)
    assert np.allclose(g2.sum(axis=1), want, rtol=1e-12)
    # q = 0 (with q = 0 exactly the acoustic Z vanish, so use the unscaled rotation instead)
    eps, U = elph.electron_bands(k, mat)
    G = elph.coupling_stage2(elph.coupling_stage1(k[0], mat, U[0]), np.zeros((1, 3)), mat)[0]
    gz = elph.rotate_final(G, U[0], np.eye(3))                            # (m', n, s)
    diag = np.einsum("mms->ms", gz)
    assert np.allclose(diag, eps[0][:, None] * c[None, :], atol=1e-13)
    off = gz.copy()
    for m in range(mat.nw):
        off[m, m] = 0
    assert np.max(np.abs(off)) < 1e-13


def test_gauge_invariance(toy):
    # Sec. 3.2: eigenvector phases are arbitrary; |g|^2 must not depend on them, and sums over
    # degenerate phonon subspaces are invariant under unitary mixing inside them.
    mat, _ = toy
    rng = np.random.default_rng(7)
    k = rng.uniform(0, 1, 3)
    q = np.array([0.25, 0.25, 0.5])        # toy modes x and y are degenerate here
    eps_k, U_k = elph.electron_bands(k[None], mat)
    eps_kq, U_kq = elph.electron_bands((k + q)[None], mat)
    om, z = elph.phonon_modes(q[None], mat)
    G = elph.coupling_stage2(elph.coupling_stage1(k, mat), q[None], mat)       # (1, m, n, s)
    Zq = elph.mode_factors(om, z, mat.mass_amu, 1e-4)
    ref = np.abs(elph.bloch_coupling(G, U_kq, U_k, Zq)) ** 2
    ph1 = np.exp(1j * rng.uniform(0, 2 * np.pi, mat.nw))
    ph2 = np.exp(1j * rng.uniform(0, 2 * np.pi, mat.nw))
    # mix the degenerate phonon pair with a random 2x2 unitary
    deg = np.nonzero(np.abs(om[0] - om[0][0]) < 1e-9)[0]
    assert len(deg) == 2
    X = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    Wu, _ = np.linalg.qr(X)
    z2 = z.copy()
    z2[0][:, deg] = z[0][:, deg] @ Wu
    Z2 = elph.mode_factors(om, z2, mat.mass_amu, 1e-4)
    got = np.abs(elph.bloch_coupling(G, U_kq * ph1, U_k * ph2, Z2)) ** 2
    others = [v for v in range(3) if v not in deg]
    assert np.allclose(got[..., others], ref[..., others], rtol=1e-12)
    assert np.allclose(got[..., deg].sum(-1), ref[..., deg].sum(-1), rtol=1e-12)
    assert not np.allclose(got[..., deg], ref[..., deg], rtol=1e-6)


def _einstein_closed_form(eps_k, eps_all, hw0, g0sq, T, mu, sigma, cut):
    kT = 8.617333262e-5 * T
    n0 = 1.0 / (np.exp(hw0 / kT) - 1.0)
    f = 1.0 / (np.exp((eps_all - mu) / kT) + 1.0)

    def dlt(x):
        return np.where(np.abs(x) < cut * sigma, np.exp(-(x / sigma) ** 2) / (np.sqrt(np.pi) * sigma), 0.0)
    out = []
    for e in eps_k:
        s = (n0 + 1 - f) * dlt(e - hw0 - eps_all) + (n0 + f) * dlt(e + hw0 - eps_all)
        out.append(2 * np.pi * g0sq * s.mean())
    return np.array(out)


def test_closed_form_einstein_linewidth():
    # Sec. 4.2 Eq. 29 for one tight-binding band, an Einstein mode (D = lam I) and constant g:
    # sum_nu |g_nu|^2 = |c|^2 hbar^2/(2 M hbar w0) = g0^2 and
    # Gamma_k = 2 pi g0^2 (1/N) sum_k' [(n0+1-f') d(e_k - w0 - e_k') + (n0+f') d(e_k + w0 - e_k')]
    # i.e. a smeared density of states at e_k -+ hbar w0, computed here from eps(k') alone.
    lam, M, cvec, n = 0.215, 28.0, np.array([0.3, -0.2, 0.1]), 8
    mat, prm = W.tb_einstein(eps0=0.05, t=0.25, lam=lam, c=cvec, mass=M, n=n, mu=0.1)
    ks, bs, gam = elph.linewidths_rta(mat, prm)
    hw0 = HBAR * np.sqrt(EV / (ANG ** 2 * AMU)) / EV * np.sqrt(lam)
    g0sq = np.sum(cvec ** 2) * (HBAR ** 2 / (AMU * EV * ANG ** 2)) / (2 * M * hw0)
    idx = np.indices((n, n, n)).reshape(3, -1).T / n
    eps_all = 0.05 - 2 * 0.25 * np.sum(np.cos(2 * np.pi * idx), axis=1)
    want = _einstein_closed_form(eps_all, eps_all, hw0, g0sq, prm.T_K, prm.mu_eV, prm.sigma_eV,
                                 prm.delta_cut_sigmas)
    assert np.array_equal(ks, np.arange(n ** 3))
    assert np.allclose(gam, want, rtol=1e-11, atol=1e-14)
    assert np.max(gam) > 1e-3
    # Gamma depends on k only through eps_k: invariant under k -> -k and axis permutations
    i = np.indices((n, n, n)).reshape(3, -1).T
    flip = ((-i[:, 0] % n) * n + (-i[:, 1] % n)) * n + (-i[:, 2] % n)
    perm = (i[:, 1] * n + i[:, 2]) * n + i[:, 0]
    assert np.allclose(gam[flip], gam, rtol=1e-11)
    assert np.allclose(gam[perm], gam, rtol=1e-11)


def test_gamma_nonnegative_and_quadratic_in_g(toy):
    mat, prm = toy
    ks, bs, g1 = elph.linewidths_rta(mat, prm, k_indices=[3, 100])
    mat2 = W.Material(**{**mat.__dict__, "g": 1.7 * mat.g})
    _, _, g2 = elph.linewidths_rta(mat2, prm, k_indices=[3, 100])
    assert np.all(g1 >= 0)
    assert np.allclose(g2, 1.7 ** 2 * g1, rtol=1e-13)


def test_degenerate_average_is_gauge_invariant():
    # Two identical copies of a band: every k is doubly degenerate; raw Gamma per band depends
    # on the basis chosen inside the pair, their average (the reading for degenerate bands) not.
    base, prm = W.tb_einstein(eps0=0.05, t=0.25, n=4, mu=0.1)
    rng = np.random.default_rng(8)
    H = np.zeros((len(base.R_H), 2, 2), dtype=np.complex128)
    H[:, 0, 0] = base.H[:, 0, 0]
    H[:, 1, 1] = base.H[:, 0, 0]
    g = (rng.normal(size=(1, 1, 2, 2, 3)) + 1j * rng.normal(size=(1, 1, 2, 2, 3))) * 0.2
    mat = W.Material("deg", 2, 1, base.mass_amu, base.lattice, base.positions, base.R_H, base.w_H, H,
                     base.R_fc, base.w_fc, base.Phi, base.Re, base.we, base.Rp, base.wp, g)
    tab = elph.electron_table(mat, prm)
    F, eps_F, U_F, k2F = tab
    ks, bs, avg, raw = elph.linewidths_rta(mat, prm, return_raw=True, table=tab)
    U2 = U_F.copy()
    for i in range(len(U2)):
        X = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
        Q, _ = np.linalg.qr(X)
        U2[i] = U_F[i] @ Q
    ks2, bs2, avg2, raw2 = elph.linewidths_rta(mat, prm, return_raw=True, table=(F, eps_F, U2, k2F))
    assert np.allclose(avg, avg2, rtol=1e-12)
    assert not np.allclose(raw, raw2, rtol=1e-6)


def test_inverse_transform_round_trip(toy):
    # Eqs. 12-13 are a transform pair: Bloch couplings on the coarse 3^3 grids, transformed back
    # with e^{-i(k.Re + q.Rp)}/(N_k N_q) and the inverse rotations, recover g(Re,Rp) on the full
    # 3^3 supercell set {-1,0,1}^3 (here with the unscaled eigenvectors z, as Eq. 12 does).
    mat, _ = toy
    pts = elph.grid_points((3, 3, 3))
    N = len(pts)
    kk = np.repeat(pts, N, axis=0)
    qq = np.tile(pts, (N, 1))
    eps_k, U_k = elph.electron_bands(kk, mat)
    eps_kq, U_kq = elph.electron_bands(kk + qq, mat)
    om, z = elph.phonon_modes(qq, mat)
    GW = np.empty((len(kk), 2, 2, 3), dtype=np.complex128)
    for p in range(len(kk)):
        GW[p] = elph.coupling_stage2(elph.coupling_stage1(kk[p], mat), qq[p:p + 1], mat)[0]
    gB = elph.bloch_coupling(GW, U_kq, U_k, z)                         # g0 in the Bloch basis
    # inverse: G^W = U_{k+q} g0 U_k^dagger z^{-1}, then the inverse Fourier sum
    back = np.einsum("pmb,pbcs,pnc->pmns", U_kq, gB, np.conj(U_k))
    back = np.einsum("pmnv,psv->pmns", back, np.conj(z))
    ph = np.exp(-2j * np.pi * (kk @ mat.Re.T.astype(float)))[:, :, None] * \
        np.exp(-2j * np.pi * (qq @ mat.Rp.T.astype(float)))[:, None, :]   # (p, Re, Rp)
    rec = np.einsum("pab,pmns->abmns", ph, back) / (N * N)
    assert np.allclose(rec, mat.g, atol=1e-13)


def test_energy_window_selects_initial_states_only():
    # Sec. 5.2: energy window |eps - mu| < cutoff on the initial states (strict)
    eps = np.array([[-1.0, -0.2, 0.5, 0.9], [0.1, 0.49999, 0.50001, 2.0]])
    ks, bs = elph.active_states(eps, 0.0, 0.5)
    assert list(zip(ks, bs)) == [(0, 1), (1, 0), (1, 1)]
    ks, bs = elph.active_states(eps, 0.0, 0.0)
    assert len(ks) == 8


def test_dead_modes_contribute_nothing(toy):
    # Reading for zero modes: hbar omega < omega_cut contributes 0 (their |g|^2 n diverges)
    mat, prm = toy
    om, z = elph.phonon_modes(np.array([[0.0, 0.25, 0.5]]), mat)
    Z = elph.mode_factors(om, z, mat.mass_amu, 1e-4)
    assert om[0, 0] < 1e-6 and np.all(Z[0][:, 0] == 0)
    assert np.all(np.linalg.norm(Z[0][:, 1:], axis=0) > 0)
    _, _, g = elph.linewidths_rta(mat, prm.with_(omega_cut_eV=1.0), k_indices=[5])
    assert np.all(g == 0.0)


def test_oracle_reproduces_stored_toy_values(toy):
    # regression pin of the oracle against its committed output (tests/golden/make_golden.py)
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "toy_seed0_gamma.txt")
    ref = np.loadtxt(path)
    mat, prm = toy
    ks, bs, gam = elph.linewidths_rta(mat, prm)
    assert np.array_equal(ref[:, 0].astype(int), ks) and np.array_equal(ref[:, 1].astype(int), bs)
    assert np.allclose(gam, ref[:, 2], rtol=1e-12, atol=0)


def test_population_window_is_an_energy_window():
    # Sec. 5.2 population window f(1-f) > delta: with f(1-f) = 1/(4 cosh^2(x/2)), x = (e - mu)/kT, it keeps
    # exactly |e - mu| < 2 kT acosh(1/(2 sqrt(delta)))
    rng = np.random.default_rng(12)
    eps = rng.uniform(-0.6, 0.6, (300, 4))
    T, mu, delta = 300.0, 0.05, 1e-3
    W = 2 * elph.KB_EV * T * np.arccosh(1 / (2 * np.sqrt(delta)))
    far = np.abs(np.abs(eps - mu) - W) > 1e-9
    eps = np.where(far, eps, mu + 2 * W)
    k1, b1 = elph.active_states(eps, mu, 0.0, T, delta)
    k2, b2 = elph.active_states(eps, mu, W)
    assert np.array_equal(k1, k2) and np.array_equal(b1, b2)
    assert 0 < len(k1) < eps.size


def test_closed_form_einstein_phonon_rate():
    # Sec. 4.3 phonon-electron rate for one tight-binding band, an Einstein mode (three
    # degenerate modes, averaged) and constant g: with sum_nu |g_nu|^2 = g0^2,
    # P_q = (1/3)(2 pi/N) n0 (n0+1) hbar w0 g0^2 sum_k [f(1-f)/kT]_k d(e_k - e_{k+q} - hbar w0),
    # computed here from eps(k) on the integer grid alone.
    lam, M, cvec, n = 0.215, 28.0, np.array([0.3, -0.2, 0.1]), 8
    mat, prm = W.tb_einstein(eps0=0.05, t=0.25, lam=lam, c=cvec, mass=M, n=n, mu=0.1)
    P = elph.phonon_rates_elph(mat, prm)
    hw0 = HBAR * np.sqrt(EV / (ANG ** 2 * AMU)) / EV * np.sqrt(lam)
    g0sq = np.sum(cvec ** 2) * (HBAR ** 2 / (AMU * EV * ANG ** 2)) / (2 * M * hw0)
    kT = 8.617333262e-5 * prm.T_K
    n0 = 1.0 / np.expm1(hw0 / kT)
    i = np.indices((n, n, n)).reshape(3, -1).T
    eps = 0.05 - 2 * 0.25 * np.sum(np.cos(2 * np.pi * i / n), axis=1)
    f = 1.0 / (np.exp((eps - 0.1) / kT) + 1.0)
    s, cut = prm.sigma_eV, prm.delta_cut_sigmas
    want = np.zeros(n ** 3)
    for iq, j in enumerate(i):
        kq = (i + j) % n
        e_kq = eps[(kq[:, 0] * n + kq[:, 1]) * n + kq[:, 2]]
        x = eps - e_kq - hw0
        d = np.where(np.abs(x) < cut * s, np.exp(-(x / s) ** 2) / (np.sqrt(np.pi) * s), 0.0)
        want[iq] = 2 * np.pi / n ** 3 * n0 * (n0 + 1) * hw0 * g0sq / 3.0 * np.sum(f * (1 - f) / kT * d)
    assert P.shape == (n ** 3, 3)
    assert np.allclose(P, want[:, None], rtol=1e-11, atol=1e-16)
    assert np.max(P) > 1e-5


def test_phonon_rate_nonnegative_and_quadratic_in_g(toy):
    mat, prm = toy
    p1 = elph.phonon_rates_elph(mat, prm)
    mat2 = W.Material(**{**mat.__dict__, "g": 1.3 * mat.g})
    p2 = elph.phonon_rates_elph(mat2, prm)
    assert np.all(p1 >= 0) and np.max(p1) > 0
    assert np.allclose(p2, 1.3 ** 2 * p1, rtol=1e-12)
    # the three acoustic modes at Gamma are dead (omega < omega_cut): no rate
    assert np.all(p1[0] == 0.0)


def test_closed_form_einstein_linewidth_adaptive_smearing():
    # Sec. 4.7 adaptive Gaussian smearing on the Einstein model: with a = 1 A (simple cubic) the
    # band velocity is hbar v_a = 2t sin(2 pi k_a + phi), b_beta = 2 pi e_beta, so each pair (k, k')
    # has sigma = max((1/sqrt 12)(2 pi/N)|v(k) - v(k')|, sigma_min), and Gamma_k is the smeared DOS
    # sum of the fixed-width closed form with that width per pair, all from eps(k) and v(k) alone.
    lam, M, cvec, n, t, phi = 0.215, 28.0, np.array([0.3, -0.2, 0.1]), 8, 0.25, 0.3
    mat, prm = W.tb_einstein(eps0=0.05, t=t, lam=lam, c=cvec, mass=M, n=n, mu=0.1, hop_phase=phi)
    prm = prm.with_(smearing=1, sigma_min_eV=2e-3)
    ks, bs, gam = elph.linewidths_rta(mat, prm)
    hw0 = HBAR * np.sqrt(EV / (ANG ** 2 * AMU)) / EV * np.sqrt(lam)
    g0sq = np.sum(cvec ** 2) * (HBAR ** 2 / (AMU * EV * ANG ** 2)) / (2 * M * hw0)
    kT = 8.617333262e-5 * prm.T_K
    n0 = 1.0 / np.expm1(hw0 / kT)
    x = np.indices((n, n, n)).reshape(3, -1).T / n
    eps = 0.05 - 2 * t * np.sum(np.cos(2 * np.pi * x + phi), axis=1)
    vel = 2 * t * np.sin(2 * np.pi * x + phi)
    f = 1.0 / (np.exp((eps - 0.1) / kT) + 1.0)
    cut = prm.delta_cut_sigmas
    want = np.zeros(n ** 3)
    for i in range(n ** 3):
        sg = np.maximum(2 * np.pi / n * np.linalg.norm(vel[i] - vel, axis=1) / np.sqrt(12.0), 2e-3)

        def dlt(y):
            return np.where(np.abs(y) < cut * sg, np.exp(-(y / sg) ** 2) / (np.sqrt(np.pi) * sg), 0.0)
        s = (n0 + 1 - f) * dlt(eps[i] - hw0 - eps) + (n0 + f) * dlt(eps[i] + hw0 - eps)
        want[i] = 2 * np.pi * g0sq * s.mean()
    assert np.array_equal(ks, np.arange(n ** 3))
    assert np.allclose(gam, want, rtol=1e-10, atol=1e-14)
    fixed = elph.linewidths_rta(mat, prm.with_(smearing=0))[2]
    assert not np.allclose(gam, fixed, rtol=1e-3)          # the width really varies per pair


def test_adaptive_sigma_scaling():
    # the width is the energy change across one mesh cell: it halves when the mesh doubles and
    # is symmetric in the two states; a rotated lattice leaves it unchanged with rotated velocities
    rng = np.random.default_rng(9)
    lat = rng.normal(size=(3, 3)) + 3 * np.eye(3)
    va, vb = rng.normal(size=(5, 3)), rng.normal(size=(5, 3))
    s8 = elph.adaptive_sigma(va, vb, lat, (8, 8, 8), 0.0)
    assert np.allclose(elph.adaptive_sigma(va, vb, lat, (16, 16, 16), 0.0), s8 / 2, rtol=1e-13)
    assert np.allclose(elph.adaptive_sigma(vb, va, lat, (8, 8, 8), 0.0), s8, rtol=1e-13)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    assert np.allclose(elph.adaptive_sigma(va @ Q, vb @ Q, lat @ Q, (8, 8, 8), 0.0), s8, rtol=1e-12)
    assert np.all(elph.adaptive_sigma(va, va, lat, (8, 8, 8), 1e-3) == 1e-3)


def test_closed_form_einstein_linewidth_final_state_window():
    # Sec. 5.2 windows on both states of a transition (window_final = 1): the Einstein closed form
    # with the sum over k' restricted to |e_k' - mu| < window; initial states are those in the window.
    lam, M, cvec, n, win = 0.215, 28.0, np.array([0.3, -0.2, 0.1]), 8, 0.43   # no energy on the edge
    mat, prm = W.tb_einstein(eps0=0.05, t=0.25, lam=lam, c=cvec, mass=M, n=n, mu=0.1)
    prm = prm.with_(window_eV=win, window_final=1)
    ks, bs, gam = elph.linewidths_rta(mat, prm)
    hw0 = HBAR * np.sqrt(EV / (ANG ** 2 * AMU)) / EV * np.sqrt(lam)
    g0sq = np.sum(cvec ** 2) * (HBAR ** 2 / (AMU * EV * ANG ** 2)) / (2 * M * hw0)
    idx = np.indices((n, n, n)).reshape(3, -1).T / n
    eps_all = 0.05 - 2 * 0.25 * np.sum(np.cos(2 * np.pi * idx), axis=1)
    inside = np.abs(eps_all - 0.1) < win
    assert np.array_equal(ks, np.nonzero(inside)[0]) and 0 < inside.sum() < n ** 3
    kT = 8.617333262e-5 * prm.T_K
    n0 = 1.0 / np.expm1(hw0 / kT)
    f = 1.0 / (np.exp((eps_all - 0.1) / kT) + 1.0)
    s, cut = prm.sigma_eV, prm.delta_cut_sigmas

    def dlt(x):
        return np.where(np.abs(x) < cut * s, np.exp(-(x / s) ** 2) / (np.sqrt(np.pi) * s), 0.0)
    want = []
    for e in eps_all[inside]:
        t = ((n0 + 1 - f) * dlt(e - hw0 - eps_all) + (n0 + f) * dlt(e + hw0 - eps_all)) * inside
        want.append(2 * np.pi * g0sq * t.mean())
    assert np.allclose(gam, want, rtol=1e-11, atol=1e-14)
    wide = elph.linewidths_rta(mat, prm.with_(window_final=0))[2]
    assert np.all(gam <= wide + 1e-15) and np.any(gam < wide - 1e-6)   # edge states lose transitions


def _polar_si(alpha=1.0):
    mat, prm = W.si_like(seed=0, nk=4)
    zs = np.diag([2.0, 2.2, 1.8])
    return mat, prm, {"Zstar": np.stack([zs, -zs]), "eps_inf": np.array([[9.0, 0.5, 0.0], [0.5, 10.0, 0.2],
                                                                        [0.0, 0.2, 11.0]]), "alpha": alpha}


def test_coulomb_constant():
    e, eps0 = 1.602176634e-19, 8.8541878128e-12          # CODATA 2018
    assert elph.E2_4PI_EPS0_EV_A == pytest.approx(e / (4 * np.pi * eps0) * 1e10, rel=1e-12)


def test_polar_long_range_small_q_limit():
    # Sec. 3.2 Eq. polarlong: as q -> 0 only the G = 0 term diverges, so for the optical modes
    # |q| L_q -> i (4 pi/V) e^2/(4 pi eps0) sum_s (qhat . Z*_s . Zq_s) / (qhat . eps . qhat)
    mat, prm, pol = _polar_si()
    A = mat.lattice
    B = 2 * np.pi * np.linalg.inv(A).T
    V = abs(np.linalg.det(A))
    direction = np.array([0.3, -0.2, 0.5])
    errs = []
    for d in (1e-3, 1e-4):
        q = d * direction[None, :]
        om, z = elph.phonon_modes(q, mat)
        Zq = elph.mode_factors(om, z, mat.mass_amu, prm.omega_cut_eV)
        L = elph.polar_long_range(q, mat, pol, Zq)[0]
        qc = q[0] @ B
        qh = qc / np.linalg.norm(qc)
        want = np.zeros(6, dtype=complex)
        for s in range(2):
            want += (qh @ pol["Zstar"][s]) @ Zq[0, 3 * s:3 * s + 3, :]
        want *= 1j * 4 * np.pi / V * elph.E2_4PI_EPS0_EV_A / (qh @ pol["eps_inf"] @ qh)
        got = np.linalg.norm(qc) * L
        errs.append(np.max(np.abs(got[3:] - want[3:])) / np.max(np.abs(want[3:])))
    assert errs[1] < 1e-3 and errs[1] < errs[0] / 5          # converges linearly in |q|


def test_polar_long_range_scalings():
    # linear in Z*; unchanged under eps -> c eps with alpha -> c alpha up to 1/c; a dead mode gives 0
    mat, prm, pol = _polar_si()
    q = np.array([[0.25, 0.0, 0.5], [0.1, 0.2, 0.3]])
    om, z = elph.phonon_modes(q, mat)
    Zq = elph.mode_factors(om, z, mat.mass_amu, prm.omega_cut_eV)
    L = elph.polar_long_range(q, mat, pol, Zq)
    L2 = elph.polar_long_range(q, mat, {**pol, "Zstar": 1.5 * pol["Zstar"]}, Zq)
    assert np.allclose(L2, 1.5 * L, rtol=1e-12)
    L3 = elph.polar_long_range(q, mat, {**pol, "eps_inf": 2 * pol["eps_inf"], "alpha": 2.0}, Zq)
    assert np.allclose(L3, L / 2, rtol=1e-10)
    Zd = Zq.copy()
    Zd[:, :, 4] = 0.0
    assert np.all(elph.polar_long_range(q, mat, pol, Zd)[:, 4] == 0)
    assert np.max(np.abs(L)) > 1e-3


def test_polar_coupling_adds_coherently():
    # g = g^S + L_q [U_{k+q}^dagger U_k]: doubling L (Z* -> 2 Z*) with g^S = 0 quadruples Gamma
    mat, prm, pol = _polar_si()
    mat0 = W.Material(**{**mat.__dict__, "g": 0.0 * mat.g})
    ks, bs, g1 = elph.linewidths_rta(mat0, prm, k_indices=[0, 5], polar=pol)
    _, _, g2 = elph.linewidths_rta(mat0, prm, k_indices=[0, 5], polar={**pol, "Zstar": 2 * pol["Zstar"]})
    assert np.all(g1 > 0) and np.allclose(g2, 4 * g1, rtol=1e-10)
    _, _, gs = elph.linewidths_rta(mat, prm, k_indices=[0, 5])
    _, _, gt = elph.linewidths_rta(mat, prm, k_indices=[0, 5], polar=pol)
    assert not np.allclose(gt, gs + g1, rtol=1e-3)           # interference between g^S and g^L


def test_three_phonon_einstein_closed_form():
    # Sec. 4.3 with two Einstein atoms (hbar w2 = 2 hbar w1) and on-site third-order constants:
    # every q contributes alike.  Modes at w1 coalesce with a w1 mode into a w2 mode, modes at w2
    # decay into two w1 modes; averaged over the degenerate modes,
    #   A(w1) = 2 pi (1/3) sum |Phi3[0a,0b,1c]|^2 c1^2 c2 n1 n1 (n2+1) / (sqrt(pi) sigma)
    #   A(w2) = 2 pi (1/3) sum |Phi3[1a,0b,0c]|^2 c2 c1^2 (1/2) n2 (n1+1)^2 / (sqrt(pi) sigma)
    # with c = hbar^2 / (2 M hbar w) from Eq. 7's mode factor.
    mat, anh, prm = W.einstein3(lam1=0.1, mass1=28.0, mass2=20.0, n=4)
    A = elph.three_phonon_diag(mat, anh, prm)
    hw1 = HBAR * np.sqrt(EV / (ANG ** 2 * AMU)) / EV * np.sqrt(0.1)
    hw2 = 2 * hw1
    h2 = HBAR ** 2 / (AMU * EV * ANG ** 2)
    c1, c2 = h2 / (2 * 28.0 * hw1), h2 / (2 * 20.0 * hw2)
    kT = 8.617333262e-5 * prm.T_K
    n1, n2 = 1 / np.expm1(hw1 / kT), 1 / np.expm1(hw2 / kT)
    d0 = 1 / (np.sqrt(np.pi) * prm.sigma_eV)
    P = anh.Phi3[0]
    a1 = 2 * np.pi / 3 * np.sum(P[:3, :3, 3:] ** 2) * c1 ** 2 * c2 * n1 * n1 * (n2 + 1) * d0
    a2 = 2 * np.pi / 3 * np.sum(P[3:, :3, :3] ** 2) * c2 * c1 ** 2 * 0.5 * n2 * (n1 + 1) ** 2 * d0
    assert np.allclose(A[:, :3], a1, rtol=1e-11) and np.allclose(A[:, 3:], a2, rtol=1e-11)


def test_three_phonon_phase_convention():
    # one off-site pair (R0, R0'): with q-independent Einstein modes V3 = e^{-i 2 pi (q.R0 + q'.R0')} C
    R0, R0p = (1, 0, 0), (0, 1, 0)
    mat, anh, prm = W.einstein3(offsite=(R0, R0p))
    rng = np.random.default_rng(11)
    q, qp, qpp = rng.uniform(0, 1, (3, 5, 3))
    V = elph.v3_coupling(q, qp, qpp, mat, anh)
    V0 = elph.v3_coupling(np.zeros((1, 3)), np.zeros((1, 3)), np.zeros((1, 3)), mat, anh)[0]
    ph = np.exp(-2j * np.pi * (q @ np.array(R0, float) + qp @ np.array(R0p, float)))
    assert np.allclose(V, ph[:, None, None, None] * V0[None], rtol=1e-12, atol=1e-15)
    wrong = np.exp(+2j * np.pi * (q @ np.array(R0, float) + qp @ np.array(R0p, float)))
    assert not np.allclose(V, wrong[:, None, None, None] * V0[None], rtol=1e-3)


def test_three_phonon_factorised_equals_brute_force():
    # the grid form (R sum at fixed q, then R' over all q~) equals the direct definition on a 3^3 grid
    mat, anh, prm = W.three_phonon_si_like(seed=1, nq=3)
    prm = prm.with_(sigma_eV=0.02)
    A = elph.three_phonon_diag(mat, anh, prm, q_indices=[1, 5])
    qs = elph.grid_points((3, 3, 3))
    om, z = elph.phonon_modes(qs, mat)
    nB = elph.bose_einstein(om, prm.T_K)
    alive = om >= prm.omega_cut_eV
    for row, iq in enumerate([1, 5]):
        acc = np.zeros(6)
        for it in range(27):
            qpp = qs[iq] + qs[it]
            i2 = elph.grid_index(qpp[None, :], (3, 3, 3))[0]
            V = elph.v3_coupling(qs[iq][None], qs[it][None], -qpp[None], mat, anh)[0]
            for nu in range(6):
                for a in range(6):
                    for b in range(6):
                        if not (alive[iq, nu] and alive[it, a] and alive[i2, b]):
                            continue
                        d1 = elph.gaussian_delta(np.array(om[iq, nu] + om[it, a] - om[i2, b]), 0.02, 6.0)
                        d2 = elph.gaussian_delta(np.array(om[iq, nu] - om[it, a] - om[i2, b]), 0.02, 6.0)
                        acc[nu] += abs(V[nu, a, b]) ** 2 * (nB[iq, nu] * nB[it, a] * (nB[i2, b] + 1) * d1
                                                            + 0.5 * nB[iq, nu] * (nB[it, a] + 1) * (nB[i2, b] + 1) * d2)
        acc *= 2 * np.pi / 27
        want = acc.copy()
        for nu in range(6):
            grp = np.abs(om[iq] - om[iq, nu]) < prm.degen_tol_eV
            want[nu] = acc[grp].mean()
        assert np.allclose(A[row], want, rtol=1e-9, atol=1e-18)
    assert np.max(A) > 0
