"""Pins of the learned-proposal oracle (CPU only).

The learned proposal is not in the paper; it samples the q sum of Eq. 29
(Sec. 4.2).  Each test below checks the oracle against something other than
itself: published test vectors, an independent library rounding, finite
differences, a closed form, or an exact property of the estimator.
"""
import numpy as np
import pytest

from oracle import elph
from oracle import sampler as S
from workloads import synthetic as W

HBAR = 1.054571817e-34
EV = 1.602176634e-19
AMU = 1.66053906660e-27
ANG = 1e-10


def test_philox_published_test_vectors():
    # Known-answer vectors of Philox4x32-10 published with the generator (Random123 distribution)
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in cases:
        got = S.philox4x32_10(np.array([ctr], dtype=np.uint64), key)[0]
        assert tuple(int(x) for x in got) == want


def test_is_uniforms_range_and_moments():
    u = S.is_uniforms(seed=12345, k_index=7, n=200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / len(u))
    assert abs(np.var(u) - 1 / 12) < 2e-3
    assert not np.array_equal(u[:100], S.is_uniforms(seed=12345, k_index=8, n=100))
    assert np.array_equal(u[:100], S.is_uniforms(seed=12345, k_index=7, n=100))


def test_bf16_round_matches_library_rounding():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(10000).astype(np.float32) * 3
    x[:3] = [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8]      # ties go to even
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.bf16_round(x), want)
    assert S.bf16_round(np.float32([1.0 + 2.0 ** -8]))[0] == 1.0
    assert S.bf16_round(np.float32([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


def _random_blob(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    th = {}
    for name, shape in S.SHAPES:
        fan_in = shape[1] if len(shape) == 2 else S.NH
        th[name] = rng.uniform(-1, 1, shape) * scale / np.sqrt(fan_in)
    return S.pack(th).astype(np.float32)


def test_mlp_gradient_matches_finite_differences():
    # backward pass (chain rule) against central differences of the FP64 loss
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, (60, S.NIN))
    off = np.array([0, 25, 60])
    t = rng.uniform(0, 1, 60) ** 4
    theta = S.bf16_params(_random_blob(2, scale=2.0))

    def loss_of(th):
        z, _ = S.mlp_forward(th, X)
        return S.softmax_ce(z, off, t)[0]

    z, cache = S.mlp_forward(theta, X)
    _, dz = S.softmax_ce(z, off, t)
    g = S.mlp_backward(theta, cache, dz)
    h = 1e-6
    for name, shape in S.SHAPES:
        flat = theta[name].ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            tp = {k: v.copy() for k, v in theta.items()}
            tm = {k: v.copy() for k, v in theta.items()}
            tp[name].ravel()[idx] += h
            tm[name].ravel()[idx] -= h
            fd = (loss_of(tp) - loss_of(tm)) / (2 * h)
            an = g[name].ravel()[idx]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(fd)), (name, idx, fd, an)


def test_softmax_ce_minimum_and_gradient_sum():
    # the cross entropy is minimal (= entropy of t, gradient 0) when softmax(z) = t
    rng = np.random.default_rng(3)
    t = rng.uniform(0.1, 1, 40)
    off = np.array([0, 15, 40])
    z = np.log(t.copy())
    z[15:] += 3.0                          # a constant shift per group changes nothing
    loss, dz = S.softmax_ce(z, off, t)
    ent = sum(-np.sum(tt / tt.sum() * np.log(tt / tt.sum())) for tt in (t[:15], t[15:])) / 2
    assert loss == pytest.approx(ent, rel=1e-12)
    assert np.max(np.abs(dz)) < 1e-15
    loss2, dz2 = S.softmax_ce(rng.standard_normal(40), off, t)
    assert loss2 > loss
    assert abs(dz2[:15].sum()) < 1e-15 and abs(dz2[15:].sum()) < 1e-15


def test_velocities_are_band_slopes():
    # Hellmann-Feynman on Eq. 10: v = (1/2 pi) d eps / d k, checked by central differences of eigh
    mat, _ = W.toy(seed=0)
    k = np.random.default_rng(4).uniform(0, 1, (12, 3))
    eps, U = elph.electron_bands(k, mat)
    v = S.band_velocities(k, mat, U)
    h = 1e-6
    for i in range(3):
        dk = np.zeros(3)
        dk[i] = h
        ep, _ = elph.electron_bands(k + dk, mat)
        em, _ = elph.electron_bands(k - dk, mat)
        assert np.allclose(v[:, :, i], (ep - em) / (2 * h) / (2 * np.pi), rtol=1e-6, atol=1e-8)


def test_velocities_tight_binding_closed_form():
    # eps = eps0 - 2t sum cos(2 pi k_a + phi)  =>  v_a = 2t sin(2 pi k_a + phi)
    mat, _ = W.tb_einstein(eps0=0.1, t=0.3, hop_phase=0.4)
    k = np.random.default_rng(5).uniform(0, 1, (20, 3))
    _, U = elph.electron_bands(k, mat)
    v = S.band_velocities(k, mat, U)[:, 0, :]
    assert np.allclose(v, 2 * 0.3 * np.sin(2 * np.pi * k + 0.4), atol=1e-13)


def test_contributions_closed_form_einstein():
    # per-q term of Eq. 29 for one band, an Einstein mode and constant g:
    # c_k(q) = 2 pi g0^2 [(n0+1-f(e_k+q)) d(e_k - w0 - e_k+q) + (n0+f(e_k+q)) d(e_k + w0 - e_k+q)]
    lam, M, cvec, n = 0.215, 28.0, np.array([0.3, -0.2, 0.1]), 6
    mat, prm = W.tb_einstein(eps0=0.05, t=0.25, lam=lam, c=cvec, mass=M, n=n, mu=0.1)
    ks, bs, c = elph.contributions(mat, prm, k_indices=[0, 7, 100, 215])
    hw0 = HBAR * np.sqrt(EV / (ANG ** 2 * AMU)) / EV * np.sqrt(lam)
    g0sq = np.sum(cvec ** 2) * (HBAR ** 2 / (AMU * EV * ANG ** 2)) / (2 * M * hw0)
    kT = 8.617333262e-5 * prm.T_K
    n0 = 1.0 / (np.exp(hw0 / kT) - 1.0)
    idx = np.indices((n, n, n)).reshape(3, -1).T
    sig, cut = prm.sigma_eV, prm.delta_cut_sigmas

    def dlt(x):
        return np.where(np.abs(x) < cut * sig, np.exp(-(x / sig) ** 2) / (np.sqrt(np.pi) * sig), 0.0)

    for j, ik in enumerate(ks):
        e_k = 0.05 - 2 * 0.25 * np.sum(np.cos(2 * np.pi * idx[ik] / n))
        ekq = 0.05 - 2 * 0.25 * np.sum(np.cos(2 * np.pi * ((idx[ik] + idx) % n) / n), axis=1)
        f = 1.0 / (np.exp((ekq - prm.mu_eV) / kT) + 1.0)
        want = 2 * np.pi * g0sq * ((n0 + 1 - f) * dlt(e_k - hw0 - ekq) + (n0 + f) * dlt(e_k + hw0 - ekq))
        assert np.allclose(c[j], want, rtol=1e-11, atol=1e-14)
    assert np.max(c) > 1e-3


def test_contributions_sum_to_linewidth(request):
    mat, prm = W.toy(seed=0)
    tab = elph.electron_table(mat, prm)
    ks, bs, _, raw = elph.linewidths_rta(mat, prm, k_indices=[3, 77], return_raw=True, table=tab)
    ks2, bs2, c = elph.contributions(mat, prm, k_indices=[3, 77], table=tab)
    assert np.array_equal(ks, ks2) and np.array_equal(bs, bs2)
    assert np.allclose(c.mean(axis=1), raw, rtol=1e-12)
    # explicit q lists pick the same columns
    qi = np.array([[5, 5, 400, 0], [1, 2, 3, 511]] * (len(ks) // 2))
    _, _, cq = elph.contributions(mat, prm, k_indices=[3, 77], q_indices=qi, table=tab)
    assert np.allclose(cq, np.take_along_axis(c, qi, axis=1), rtol=1e-13, atol=1e-300)


def test_inverse_cdf_draws():
    p = np.array([0.1, 0.0, 0.4, 0.25, 0.25])
    cdf = np.cumsum(p)
    # u just below / at each boundary selects the bin that ends there / the next non-empty one
    assert list(S.draw(p, np.array([0.0, 0.0999999, 0.1, 0.4999, 0.5, 0.7499, 0.75, 0.9999999]))) == \
        [0, 0, 2, 2, 3, 3, 4, 4]
    u = S.is_uniforms(seed=3, k_index=0, n=200000)
    q = S.draw(p, u)
    freq = np.bincount(q, minlength=5) / len(u)
    assert np.all(np.abs(freq - p) < 5 * np.sqrt(p * (1 - p) / len(u)) + 1e-12)
    assert cdf[-1] == pytest.approx(1.0)


def test_zero_variance_proposal_is_exact():
    # with p proportional to c the estimate equals (1/N_q) sum c for any draws
    rng = np.random.default_rng(6)
    c = rng.uniform(0, 1, 300) ** 3
    p = c / c.sum()
    q = S.draw(p, S.is_uniforms(seed=9, k_index=1, n=50))
    est = S.is_estimate(c[q][None, :], p, q)
    assert est[0] == pytest.approx(c.mean(), rel=1e-12)
    # and the uniform proposal averages the sampled terms
    pu = np.full(300, 1.0 / 300)
    qu = S.draw(pu, S.is_uniforms(seed=9, k_index=2, n=50))
    assert S.is_estimate(c[qu][None, :], pu, qu)[0] == pytest.approx(c[qu].mean(), rel=1e-12)


def test_mixture_proposal_is_normalised_and_defensive():
    rng = np.random.default_rng(7)
    logits = rng.standard_normal((3, 64)) * 4
    p = S.proposal(logits, alpha=0.1)
    assert p.sum() == pytest.approx(1.0, rel=1e-14)
    assert p.min() >= 0.1 / 64 * (1 - 1e-14)


def test_importance_sampled_linewidth_is_unbiased():
    # E[Gamma^] = Gamma: the average over 32 seeds lies within 4 standard errors of the full-grid sum,
    # for the uniform proposal and for a (random, untrained) network proposal
    mat, prm = W.toy(seed=0)
    prm = prm.with_(nk=(4, 4, 4), nq=(4, 4, 4))
    tab = elph.electron_table(mat, prm)
    kk = [1, 22, 43]
    ks, bs, exact = elph.linewidths_rta(mat, prm, k_indices=kk, table=tab)
    blob = _random_blob(11, scale=3.0)
    for uniform in (True, False):
        runs = np.array([S.linewidths_is(mat, prm, blob, 0.25, 0.1, seed, k_indices=kk, uniform=uniform,
                                         table=tab)[2] for seed in range(32)])
        mean, se = runs.mean(0), runs.std(0, ddof=1) / np.sqrt(len(runs))
        assert np.all(np.abs(mean - exact) <= 4 * se + 1e-12 * exact)
        assert np.max(se) > 0


# ------------------------------------------------------------------ shell factor of the proposal

def _two_einstein(equal_ratio: bool):
    """Two Einstein frequencies (hbar w_s = 0.0647 sqrt(lam_s)); with |c|^2/M1 = |d|^2/M2 every mode's
    sum over its three degenerate partners of |g|^2 is K / (hbar w_s) with one K for both atoms."""
    c = np.array([0.3, -0.2, 0.1])
    M = (28.0, 12.0)
    d = c * np.sqrt(M[1] / M[0]) * (1.0 if equal_ratio else 1.7)
    return W.tb_einstein2(c=tuple(c), d=tuple(d), mass=M, lam=(0.215, 0.6), n=6)


def test_shell_factor_zero_variance_on_einstein_models():
    # one band, constant coupling: c_k(q) = 2 pi / (sqrt(pi) sigma) sum_nu |g_nu|^2 W_nu(q) with W the
    # bracket of Eq. 29.  With |g_nu|^2 proportional to 1/(hbar w_nu) for every mode, c / phi is the same
    # for every q, so the shell proposal p ~ phi gives the exact q sum for any draws.  The one-frequency
    # model fixes the occupation and Gaussian weights; the two-frequency model fixes the 1/(hbar w) factor.
    for mat, prm in (W.tb_einstein(eps0=0.05, t=0.25, lam=0.215, n=6, mu=0.1), _two_einstein(True)):
        tab = elph.electron_table(mat, prm)
        kk = [0, 7, 100, 215]
        ks, bs, c = elph.contributions(mat, prm, k_indices=kk, table=tab)
        phi = S.shell_factor(mat, prm, ks, bs, table=tab)
        pos = c > 0
        assert np.all(phi[pos] > 0) and np.any(pos)
        ratio = c[pos] / phi[pos]
        assert np.max(ratio) - np.min(ratio) <= 1e-10 * np.max(ratio)
        _, _, exact = elph.linewidths_rta(mat, prm, k_indices=kk, table=tab)
        for seed in (1, 2):
            _, _, est = S.linewidths_is(mat, prm, None, 0.05, 0.1, seed, k_indices=kk, table=tab, mode="shell")
            assert np.allclose(est, exact, rtol=1e-10, atol=0)
    # unequal |c|^2 / M: the two frequencies' terms no longer share one ratio (the estimate is noisy)
    mat, prm = _two_einstein(False)
    tab = elph.electron_table(mat, prm)
    ks, bs, c = elph.contributions(mat, prm, k_indices=[7, 100], table=tab)
    phi = S.shell_factor(mat, prm, ks, bs, table=tab)
    r = c[c > 0] / phi[c > 0]
    assert np.max(r) - np.min(r) > 1e-3 * np.max(r)


def test_shell_factor_vanishes_only_where_every_term_is_cut():
    # phi > 0 wherever c > 0 (the proposal then covers every non-zero term, so the estimate is unbiased);
    # phi = 0 at some q (the delta shell excludes them), and phi is unchanged by the coupling's size
    mat, prm = W.toy(seed=0)
    tab = elph.electron_table(mat, prm)
    kk = [3, 77, 300]
    ks, bs, c = elph.contributions(mat, prm, k_indices=kk, table=tab)
    phi = S.shell_factor(mat, prm, ks, bs, table=tab)
    assert phi.shape == c.shape
    assert np.all(phi[c > 0] > 0)
    prm2 = prm.with_(sigma_eV=0.01)
    ks2, bs2, c2 = elph.contributions(mat, prm2, k_indices=kk, table=tab)
    phi2 = S.shell_factor(mat, prm2, ks2, bs2, table=tab)
    assert np.all(phi2[c2 > 0] > 0) and np.any(phi2 == 0)
    mat3 = W.Material(**{**mat.__dict__, "g": mat.g * 3.0})
    assert np.array_equal(S.shell_factor(mat3, prm2, ks2, bs2, table=tab), phi2)
    qi = np.array([[0, 5, 511], [2, 2, 100], [7, 8, 9]])
    sub = S.shell_factor(mat, prm, ks[:3], bs[:3], table=tab, q_indices=qi)
    assert np.array_equal(sub, np.take_along_axis(phi[:3], qi, axis=1))


def test_shell_proposal_is_normalised_and_defensive():
    rng = np.random.default_rng(8)
    logits = rng.standard_normal((3, 64)) * 4
    phi = rng.uniform(0, 1, (3, 64)) ** 3
    phi[:, :10] = 0.0                                   # outside every row's shell
    phi[2] = 0.0                                        # a row without any shell: left out
    lp = S.log_shell(phi)
    p = S.proposal(logits, 0.1, lp)
    assert p.sum() == pytest.approx(1.0, rel=1e-14)
    assert np.all(p[:10] == 0.0)
    sh = S.shell_proposal(lp)
    assert sh.sum() == pytest.approx(1.0, rel=1e-14)
    assert np.allclose(sh, 0.5 * (phi[0] / phi[0].sum() + phi[1] / phi[1].sum()), rtol=1e-13)
    assert np.all(p >= 0.1 * sh * (1 - 1e-14))
    assert np.all(S.proposal(logits, 0.1, np.full((3, 64), -np.inf)) == 1.0 / 64)


def test_loss_gradient_with_prior_matches_finite_differences():
    rng = np.random.default_rng(12)
    X = rng.uniform(-1, 1, (50, S.NIN))
    off = np.array([0, 20, 50])
    t = rng.uniform(0, 1, 50) ** 4
    prior = rng.normal(0, 2, 50)
    t[[3, 30]] = 0.0
    prior[[3, 30]] = -np.inf                             # zero prior weight where the target is 0
    theta = S.bf16_params(_random_blob(4, scale=2.0))

    def loss_of(th):
        return S.softmax_ce(S.mlp_forward(th, X)[0], off, t, prior)[0]

    z, cache = S.mlp_forward(theta, X)
    loss, dz = S.softmax_ce(z, off, t, prior)
    assert np.isfinite(loss) and dz[3] == 0.0 and dz[30] == 0.0
    g = S.mlp_backward(theta, cache, dz)
    h = 1e-6
    for name, shape in S.SHAPES:
        flat = theta[name].ravel()
        for idx in rng.choice(flat.size, size=min(5, flat.size), replace=False):
            tp = {k: v.copy() for k, v in theta.items()}
            tm = {k: v.copy() for k, v in theta.items()}
            tp[name].ravel()[idx] += h
            tm[name].ravel()[idx] -= h
            fd = (loss_of(tp) - loss_of(tm)) / (2 * h)
            assert abs(fd - g[name].ravel()[idx]) <= 1e-6 * max(1e-3, abs(fd)), (name, idx)
    # the minimum is at softmax(z + prior) = t
    zmin = np.where(t > 0, np.log(np.where(t > 0, t, 1.0)), 0.0) - np.where(np.isfinite(prior), prior, 0.0)
    _, dzmin = S.softmax_ce(zmin, off, t, prior)
    assert np.max(np.abs(dzmin)) < 1e-15


def test_shell_and_learned_proposals_are_unbiased():
    # E[Gamma^] = Gamma over 32 seeds for the shell proposal and the network-times-shell proposal
    mat, prm = W.toy(seed=0)
    prm = prm.with_(nk=(4, 4, 4), nq=(4, 4, 4), sigma_eV=0.1)
    tab = elph.electron_table(mat, prm)
    kk = [1, 22, 43]
    ks, bs, exact = elph.linewidths_rta(mat, prm, k_indices=kk, table=tab)
    blob = _random_blob(13, scale=3.0)
    for mode in ("shell", "learned"):
        runs = np.array([S.linewidths_is(mat, prm, blob, 0.25, 0.1, seed, k_indices=kk, table=tab,
                                         mode=mode)[2] for seed in range(32)])
        mean, se = runs.mean(0), runs.std(0, ddof=1) / np.sqrt(len(runs))
        assert np.all(np.abs(mean - exact) <= 4 * se + 1e-12 * exact)
