"""Plain FP64 CPU oracle of the el-ph RTA linewidth path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library: it reads the same seeded inputs (``workloads``) and
nothing else.

Each function follows one step of the paper (arXiv 2111.14999), in the
paper's order and notation, with numpy FP64 arithmetic.  Library primitives
used as steps: ``numpy.linalg.eigh`` (Hermitian eigenproblem), ``@`` (matrix
products), ``numpy.exp``/``expm1``.  No blocking or fusion beyond what the
equations state; the one re-association used by default (R_e sum first, then
R_p, Sec. 5.5 Eq. 71) is checked against the direct double sum of Eq. 13.

Readings of points the paper leaves open (units, dagger placement, prefactor,
delta cutoff, zero modes, window, degenerate averaging) are listed at the top
of each function that applies them.

Units: eV, Angstrom, amu.  k, q in crystal coordinates; k.R = 2 pi sum_i k_i n_i.
"""
from __future__ import annotations

import numpy as np

# Physical constants (CODATA 2018 derived), carried here as literals.
KB_EV = 8.617333262e-5                 # Boltzmann constant, eV/K
HBAR_OMEGA_EV = 0.06465415130134121    # hbar*sqrt(eV/(A^2 amu)) in eV
HBAR2_AMU_EV_A2 = 0.004180159280496722  # hbar^2/(amu eV A^2), dimensionless
E2_4PI_EPS0_EV_A = 14.399645478425668  # e^2/(4 pi eps_0) in eV A

__all__ = [
    "KB_EV", "HBAR_OMEGA_EV", "HBAR2_AMU_EV_A2",
    "grid_points", "grid_index", "phases",
    "wannier_hamiltonian", "electron_bands",
    "dynamical_matrix", "phonon_modes", "mode_factors",
    "bose_einstein", "fermi_dirac", "gaussian_delta",
    "coupling_wannier_direct", "coupling_stage1", "coupling_stage2",
    "rotate_final", "bloch_coupling", "couplings_for_pairs",
    "active_states", "fine_grid", "electron_table", "linewidths_rta", "contributions",
    "phonon_rates_elph", "adaptive_sigma", "in_window", "polar_long_range", "E2_4PI_EPS0_EV_A",
    "v3_coupling", "three_phonon_diag",
]


# ---------------------------------------------------------------- grids (Sec. 5.1)

def grid_points(n) -> np.ndarray:
    """Gamma-centred Monkhorst-Pack points k = (i1/N1, i2/N2, i3/N3).

    Sec. 5.1 (Points class): points are sorted by incrementing z, then y, then
    x, i.e. index (i1*N2 + i2)*N3 + i3.
    """
    n1, n2, n3 = (int(x) for x in n)
    out = np.empty((n1 * n2 * n3, 3))
    idx = 0
    for i1 in range(n1):
        for i2 in range(n2):
            for i3 in range(n3):
                out[idx] = (i1 / n1, i2 / n2, i3 / n3)
                idx += 1
    return out


def grid_index(frac: np.ndarray, n) -> np.ndarray:
    """Index of crystal-coordinate points on the grid n (points wrapped into [0,1))."""
    n = np.asarray(n, dtype=np.int64)
    i = np.rint(np.asarray(frac) * n).astype(np.int64) % n
    return (i[..., 0] * n[1] + i[..., 1]) * n[2] + i[..., 2]


def phases(k: np.ndarray, R: np.ndarray) -> np.ndarray:
    """e^{i k.R} with k.R = 2 pi sum_i k_i n_i (k crystal, R integer lattice coords)."""
    return np.exp(2j * np.pi * (np.asarray(k, dtype=np.float64) @ np.asarray(R, dtype=np.float64).T))


# ------------------------------------------------------- electrons (Sec. 3.2, Eqs. 10-11)

def wannier_hamiltonian(k: np.ndarray, mat) -> np.ndarray:
    """H^W_k[n][m] = sum_R w_R e^{i k.R} <0n|H|Rm>   (Sec. 3.2, Eq. 10).

    Optional per-R weights w_R (Wigner-Seitz degeneracy) multiply each term.
    """
    P = phases(np.atleast_2d(k), mat.R_H) * mat.w_H[None, :]     # (nk, nR)
    return (P @ mat.H.reshape(len(mat.R_H), -1)).reshape(P.shape[0], mat.nw, mat.nw)


def electron_bands(k: np.ndarray, mat):
    """Diagonalise H^W_k: U_k^dagger H^W_k U_k = diag(eps_k)   (Sec. 3.2, Eq. 11).

    Returns eps (nk, nw) ascending and U (nk, nw, nw) with columns = eigenvectors
    (U[m, b]: Wannier index m, band b).
    """
    Hk = wannier_hamiltonian(k, mat)
    eps, U = np.linalg.eigh(Hk)
    return eps, U


# -------------------------------------------------------- phonons (Sec. 3.1, Eqs. 3-4)

def dynamical_matrix(q: np.ndarray, mat) -> np.ndarray:
    """D[s a][s' a'](q) = sum_R w_R Phi(s a 0 | s' a' R) e^{i q.R} / sqrt(M_s M_s')   (Eq. 3).

    Reading: Eq. 3 omits the masses, yet Eq. 4 makes its eigenvalues (hbar omega)^2,
    so D is the mass-scaled matrix; the phase carries no atomic positions,
    as written in Eq. 3.
    """
    P = phases(np.atleast_2d(q), mat.R_fc) * mat.w_fc[None, :]
    nm = 3 * mat.na
    D = (P @ mat.Phi.reshape(len(mat.R_fc), -1).astype(np.complex128)).reshape(P.shape[0], nm, nm)
    m = np.repeat(np.asarray(mat.mass_amu, dtype=np.float64), 3)
    return D / np.sqrt(np.outer(m, m))[None, :, :]


def phonon_modes(q: np.ndarray, mat):
    """Diagonalise D(q): D z = (hbar omega)^2 z   (Sec. 3.1, Eq. 4).

    With D in eV/(A^2 amu), hbar omega [eV] = HBAR_OMEGA_EV * sqrt(lambda).
    Negative rounding noise at acoustic zeros is clipped to 0.
    Returns omega (nq, 3na) ascending, z (nq, 3na, 3na) columns = modes.
    """
    lam, z = np.linalg.eigh(dynamical_matrix(q, mat))
    omega = HBAR_OMEGA_EV * np.sqrt(np.clip(lam, 0.0, None))
    return omega, z


def mode_factors(omega: np.ndarray, z: np.ndarray, mass_amu: np.ndarray,
                 omega_cut: float) -> np.ndarray:
    """Z_q[s a, nu] = z_q[s a, nu] * sqrt(hbar^2 / (2 M_s hbar omega_q nu))   (Eq. 7).

    Reading: the single mass m of Eq. 7 is the mass of the displaced atom s, so
    the factor sits inside the contraction over (s, a).  Modes with
    hbar omega < omega_cut are dead: their factor is 0.  Units: Angstrom.
    """
    m = np.repeat(np.asarray(mass_amu, dtype=np.float64), 3)      # (3na,)
    alive = omega >= omega_cut
    safe = np.where(alive, omega, 1.0)
    fac = np.sqrt(HBAR2_AMU_EV_A2 / (2.0 * m[None, :, None] * safe[:, None, :]))
    return np.where(alive[:, None, :], z * fac, 0.0)


# -------------------------------------------------- statistics and smearing (Secs. 4.1, 4.2, 4.7)

def bose_einstein(omega: np.ndarray, T: float) -> np.ndarray:
    """n = 1/(e^{hbar omega / k_B T} - 1)   (Sec. 4.1).  Zero for omega = 0 entries."""
    x = np.asarray(omega) / (KB_EV * T)
    with np.errstate(divide="ignore"):
        return np.where(x > 0, 1.0 / np.expm1(np.where(x > 0, x, 1.0)), 0.0)


def fermi_dirac(eps: np.ndarray, mu: float, T: float) -> np.ndarray:
    """f = 1/(e^{(eps - mu)/k_B T} + 1)   (Sec. 4.2)."""
    x = (np.asarray(eps) - mu) / (KB_EV * T)
    with np.errstate(over="ignore"):
        return 1.0 / (np.exp(x) + 1.0)


def gaussian_delta(x: np.ndarray, sigma: float, cut_sigmas: float) -> np.ndarray:
    """delta(x) ~ e^{-x^2/sigma^2} / (sqrt(pi) sigma)   (Sec. 4.7, Eq. 61).

    Reading: the Gaussian is truncated to 0 for |x| >= cut_sigmas * sigma
    (the paper states no truncation; at 6 sigma the dropped tail is e^{-36}).
    """
    x = np.asarray(x)
    val = np.exp(-(x / sigma) ** 2) / (np.sqrt(np.pi) * sigma)
    return np.where(np.abs(x) < cut_sigmas * sigma, val, 0.0)


# ------------------------------------------------------- couplings (Sec. 3.2 Eq. 13, Sec. 5.5)

def coupling_wannier_direct(k: np.ndarray, q: np.ndarray, mat) -> np.ndarray:
    """G^W(k,q) = sum_{Re,Rp} w_e w_p e^{i k.Re + i q.Rp} g(Re,Rp)   (Eq. 13, direct double sum).

    Reading: the 1/N_e of Eq. 13 is folded into the input g(Re,Rp).
    Returns (npairs, nw(m), nw(n), 3na).
    """
    k = np.atleast_2d(k)
    q = np.atleast_2d(q)
    out = np.zeros((len(k), mat.nw, mat.nw, mat.nmodes), dtype=np.complex128)
    Pe = phases(k, mat.Re) * mat.we[None, :]
    Pp = phases(q, mat.Rp) * mat.wp[None, :]
    for p in range(len(k)):
        for ie in range(len(mat.Re)):
            for ip in range(len(mat.Rp)):
                out[p] += Pe[p, ie] * Pp[p, ip] * mat.g[ie, ip]
    return out


def coupling_stage1(k: np.ndarray, mat, U_k: np.ndarray | None = None) -> np.ndarray:
    """f~(k, Rp) = sum_Re w_e e^{i k.Re} g(Re, Rp) [U_k]   (Sec. 5.5, Eq. 71: precompute at fixed k).

    Eq. 71 folds the k-side rotation U_k into the precomputed quantity; pass
    ``U_k`` (nw, nb) to apply it to the second Wannier index (n -> b).
    Returns (nRp, nw(m), nw or nb, 3na) for one k.
    """
    Pe = phases(np.atleast_2d(k), mat.Re)[0] * mat.we
    f1 = (Pe @ mat.g.reshape(len(mat.Re), -1)).reshape(mat.g.shape[1:])
    if U_k is not None:
        f1 = np.einsum("pmns,nb->pmbs", f1, U_k)
    return f1


def coupling_stage2(f1: np.ndarray, q: np.ndarray, mat) -> np.ndarray:
    """sum_Rp w_p e^{i q.Rp} f~(k, Rp) for one k and many q (Sec. 5.5, Eq. 70, R' sum).

    f1: (nRp, ...) for one k.  Returns (nq, ...).
    """
    Pp = phases(np.atleast_2d(q), mat.Rp) * mat.wp[None, :]
    return (Pp @ f1.reshape(len(mat.Rp), -1)).reshape((Pp.shape[0],) + f1.shape[1:])


def rotate_final(G: np.ndarray, U_kq: np.ndarray, Zq: np.ndarray) -> np.ndarray:
    """g[m' b nu] = sum_{m, s a} [U_{k+q}^dagger]_{m' m} G[m][b][s a] Z_q[s a, nu]   (Eq. 13 with Eq. 7).

    Reading of the daggers: the Wannier-to-Bloch rotation is U^dagger X U as
    for H^B = U^dagger H^W U in Eq. 11; the first Wannier index (m) is the k+q
    side because Eq. 7 puts psi_{k+q} in the bra.
    Shapes: G (..., nw, nb, 3na), U_kq (..., nw, nw), Zq (..., 3na, 3na).
    """
    nb, ns = G.shape[-2], G.shape[-1]
    lead = G.shape[:-3]
    UH = np.conj(np.swapaxes(U_kq, -1, -2))
    t = UH @ G.reshape(lead + (G.shape[-3], nb * ns))               # (..., m', nb*3na)
    t = t.reshape(lead + (G.shape[-3] * nb, ns)) @ Zq                # (..., m'*nb, nu)
    return t.reshape(lead + (G.shape[-3], nb, Zq.shape[-1]))


def bloch_coupling(GW: np.ndarray, U_kq: np.ndarray, U_k: np.ndarray, Zq: np.ndarray) -> np.ndarray:
    """g_{m' n nu}(k,q) = sum [U_{k+q}^dagger]_{m' m} G^W[m][n'][s a] [U_k]_{n' n} Z_q[s a, nu].

    The full Wannier-to-Bloch rotation of Eq. 13 (all bands n), used with the
    direct double sum.  Returns (..., nw(m'), nw(n), 3na(nu)).
    """
    t = np.einsum("...mns,...nb->...mbs", GW, U_k)
    return rotate_final(t, U_kq, Zq)


def couplings_for_pairs(k: np.ndarray, q: np.ndarray, mat, omega_cut: float = 1e-4,
                        direct: bool = False):
    """|g_{m' n nu}(k,q)|^2 for explicit (k,q) pairs, plus eps_k, eps_{k+q}, omega_q.

    H(k), H(k+q) and D(q) are built and diagonalised for every pair.
    Returns g2 (npairs, nw(m'), nw(n), 3na), eps_k, eps_kq (npairs, nw), omega (npairs, 3na).
    """
    k = np.atleast_2d(np.asarray(k, dtype=np.float64))
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    eps_k, U_k = electron_bands(k, mat)
    eps_kq, U_kq = electron_bands(k + q, mat)
    omega, z = phonon_modes(q, mat)
    Zq = mode_factors(omega, z, mat.mass_amu, omega_cut)
    if direct:
        g = bloch_coupling(coupling_wannier_direct(k, q, mat), U_kq, U_k, Zq)
    else:
        g = np.empty((len(k), mat.nw, mat.nw, mat.nmodes), dtype=np.complex128)
        for p in range(len(k)):
            G = coupling_stage2(coupling_stage1(k[p], mat, U_k[p]), q[p], mat)[0]
            g[p] = rotate_final(G, U_kq[p], Zq[p])
    return np.abs(g) ** 2, eps_k, eps_kq, omega


# ------------------------------------------------------- windows (Sec. 5.2) and linewidths (Eq. 29)

def active_states(eps_k: np.ndarray, mu: float, window: float, T: float | None = None,
                  population_delta: float = 0.0):
    """Windows of Sec. 5.2 on the initial states: the energy window |eps_kb - mu| < window
    (window <= 0: all), or with population_delta > 0 the population window f(1-f) > delta.

    Reading: the window applies to initial states only; final states at k+q
    range over all bands.  Returns (k_index, band) arrays ordered by k then band.
    """
    nk, nb = eps_k.shape
    ks, bs = [], []
    for ik in range(nk):
        for b in range(nb):
            if population_delta > 0:
                f = fermi_dirac(eps_k[ik, b], mu, T)
                keep = f * (1.0 - f) > population_delta
            else:
                keep = window <= 0 or abs(eps_k[ik, b] - mu) < window
            if keep:
                ks.append(ik)
                bs.append(b)
    return np.array(ks, dtype=np.int64), np.array(bs, dtype=np.int64)


def in_window(eps: np.ndarray, params) -> np.ndarray:
    """Membership of states of energies eps in the window of Sec. 5.2 (the energy window
    |eps - mu| < window, window <= 0: all; or with population_delta > 0 the population window
    f(1-f) > delta), elementwise."""
    eps = np.asarray(eps, dtype=np.float64)
    delta = getattr(params, "population_delta", 0.0)
    if delta > 0:
        f = fermi_dirac(eps, params.mu_eV, params.T_K)
        return f * (1.0 - f) > delta
    if params.window_eV <= 0:
        return np.ones(eps.shape, dtype=bool)
    return np.abs(eps - params.mu_eV) < params.window_eV


def _final_ok(eps_kq, params):
    """Final states allowed: every band (the default reading), or with window_final = 1 only those
    inside the window (Phoebe's active band structure for both states of a transition)."""
    if getattr(params, "window_final", 0) == 1:
        return in_window(eps_kq, params)
    return np.ones(np.shape(eps_kq), dtype=bool)


def _active(eps_grid, params):
    return active_states(eps_grid, params.mu_eV, params.window_eV, params.T_K,
                         getattr(params, "population_delta", 0.0))


def fine_grid(nk, nq):
    """The grid holding every k and every k+q: per axis the finer of nk, nq (one must divide the other)."""
    out = []
    for a, b in zip(nk, nq):
        a, b = int(a), int(b)
        if max(a, b) % min(a, b) != 0:
            raise ValueError("k and q grids are not commensurate")
        out.append(max(a, b))
    return tuple(out)


def electron_table(mat, params):
    """eps and U on the fine grid, plus the k-grid -> fine-grid index map."""
    nk = tuple(int(x) for x in params.nk)
    F = fine_grid(nk, params.nq)
    eps_F, U_F = electron_bands(grid_points(F), mat)
    k_to_F = grid_index(grid_points(nk), F)
    return F, eps_F, U_F, k_to_F


def adaptive_sigma(v_a: np.ndarray, v_b: np.ndarray, lattice: np.ndarray, n, sigma_min: float) -> np.ndarray:
    """Adaptive Gaussian width for a pair of states (Sec. 4.7):
    sigma = (A / sqrt 12) sqrt( sum_beta ( sum_alpha (v^alpha_a - v^alpha_b) C_alpha,beta / N_beta )^2 ),  A = 1.

    Readings: the square inside the beta sum (the printed formula has none; a signed sum
    under the root is not a width); hbar v in eV A (Cartesian); C_alpha,beta = component alpha
    of the reciprocal lattice vector b_beta = 2 pi (A^-1)^T, so sum_alpha dv_alpha C_alpha,beta
    / N_beta is the energy change across one mesh cell along b_beta; N_beta the mesh the sum
    runs over (the q grid); a floor sigma_min keeps the width positive where the velocities
    coincide.  v_a, v_b broadcast, last axis Cartesian.
    """
    B = 2.0 * np.pi * np.linalg.inv(np.asarray(lattice, dtype=np.float64)).T     # rows b_beta
    C = B.T / np.asarray(n, dtype=np.float64)[None, :]                             # C[alpha, beta] / N_beta
    d = (np.asarray(v_a) - np.asarray(v_b)) @ C
    return np.maximum(np.sqrt(np.sum(d * d, axis=-1) / 12.0), sigma_min)


def polar_long_range(qpts: np.ndarray, mat, polar, Zq: np.ndarray) -> np.ndarray:
    """q-only factor L_{q nu} of the long-range coupling (Sec. 3.2, Eq. polarlong):
    g^L_{m' n nu}(k,q) = L_{q nu} <psi_{k+q m'}|e^{i(q+G).r}|psi_{k n}>  ~  L_{q nu} [U_{k+q}^dagger U_k]_{m' n},

    L_{q nu} = i (4 pi / V) e^2/(4 pi eps_0) sum_s sum_{G, q+G != 0}
               [(q+G) . Z*_s . z^s_{q nu} sqrt(hbar^2 / (2 M_s hbar w_{q nu}))] / [(q+G) . eps_inf . (q+G)]
               * exp(-(q+G) . eps_inf . (q+G) / (4 alpha))

    Readings: the overlap's right state is psi_{k n} (the printed ket repeats k+q) and it is
    the Wannier-gauge overlap U_{k+q}^dagger U_k (the paper's U(k+q) U^dagger(k) in its
    column convention); the Gaussian filter of the cited decomposition makes the G sum
    converge (the printed sum has none), alpha a parameter, terms with exponent >= cut
    dropped; the mode factor of Eq. 7 (mass and 1/sqrt(omega), 0 for dead modes) carries
    z and the square root, with the 1/N_q of the printed root dropped as the interpolated g
    of this path carries no 1/sqrt(N); no atomic-position phase (none is printed, and the
    dynamical matrix of Eq. 3 has none).  ``polar`` = dict(Zstar (na,3,3), eps_inf (3,3),
    alpha in 1/A^2, cut).  Zq (nq, 3na, 3na) from ``mode_factors``.  Returns (nq, 3na) complex.
    """
    A = np.asarray(mat.lattice, dtype=np.float64)
    V = abs(np.linalg.det(A))
    B = 2.0 * np.pi * np.linalg.inv(A).T                   # rows b_beta, 1/A
    Zs = np.asarray(polar["Zstar"], dtype=np.float64)     # (na, 3, 3)
    eps = np.asarray(polar["eps_inf"], dtype=np.float64)
    alpha, cut = float(polar["alpha"]), float(polar.get("cut", 25.0))
    # G box large enough for every q in the first cell: |q+G|^2 <= 4 alpha cut / eps_min
    kmax = np.sqrt(4.0 * alpha * cut / np.min(np.linalg.eigvalsh(eps)))
    nmax = [int(np.ceil(kmax / (2.0 * np.pi) * np.linalg.norm(A[i]))) + 1 for i in range(3)]
    Gi = np.array(np.meshgrid(*[np.arange(-m, m + 1) for m in nmax], indexing="ij")).reshape(3, -1).T
    out = np.zeros((len(qpts), Zq.shape[2]), dtype=np.complex128)
    na = Zs.shape[0]
    for iq, q in enumerate(np.atleast_2d(qpts)):
        K = (q[None, :] + Gi) @ B                          # (nG, 3) Cartesian q+G
        x = np.einsum("ga,ab,gb->g", K, eps, K)
        keep = (x > 1e-14) & (x / (4.0 * alpha) < cut)
        K, x = K[keep], x[keep]
        fac = np.exp(-x / (4.0 * alpha)) / x               # (nG,)
        acc = np.zeros(Zq.shape[2], dtype=np.complex128)
        for s_ in range(na):
            kz = K @ Zs[s_]                                # (nG, 3): (q+G) . Z*_s
            acc += np.einsum("g,gb,bn->n", fac, kz, Zq[iq, 3 * s_:3 * s_ + 3, :])
        out[iq] = 1j * (4.0 * np.pi / V) * E2_4PI_EPS0_EV_A * acc
    return out


def linewidths_rta(mat, params, k_indices=None, direct: bool = False, return_raw: bool = False,
                   table=None, polar=None):
    """RTA linewidths Gamma_nk = hbar/tau_nk of the active states   (Sec. 4.2 Eq. 29, Sec. 4.3.2).

    Gamma_nk = (2 pi / N_q) sum_q sum_{m' nu} |g_{m' n nu}(k,q)|^2
               [ (n_q nu + 1 - f_{m',k+q}) delta(eps_nk - hbar w_q nu - eps_{m',k+q})
               + (n_q nu + f_{m',k+q})     delta(eps_nk + hbar w_q nu - eps_{m',k+q}) ]

    Readings: the sum over k' with delta(k - k' + q) in Eq. 29 is a sum over q
    with k' = k + q (looked up on the grid, Sec. 5.1); the prefactor
    2 pi/(N_k V) becomes 2 pi/N_q with hbar = 1 energy units (Gamma in eV), no
    cell volume and no spin factor; f is the equilibrium Fermi-Dirac
    occupation; delta is the truncated Gaussian of Eq. 61; dead modes
    (hbar omega < omega_cut) contribute nothing; Gamma is finally averaged over
    active bands degenerate within degen_tol at the same k.

    ``k_indices``: optional k-grid indices restricting the initial k points.
    ``direct``: use the direct double sum of Eq. 13 instead of Eqs. 70-71.
    ``polar``: optional long-range parameters (see ``polar_long_range``); g = g^S + g^L.
    Returns (k_index, band, gamma) ordered by k index then band.
    """
    nk = tuple(int(x) for x in params.nk)
    nq = tuple(int(x) for x in params.nq)
    qpts = grid_points(nq)
    kpts = grid_points(nk)
    Nq = len(qpts)
    T, mu, sigma = params.T_K, params.mu_eV, params.sigma_eV
    cut = params.delta_cut_sigmas

    F, eps_F, U_F, k_to_F = table if table is not None else electron_table(mat, params)
    eps_grid = eps_F[k_to_F]
    ks, bs = _active(eps_grid, params)
    if k_indices is not None:
        keep = np.isin(ks, np.asarray(k_indices))
        ks, bs = ks[keep], bs[keep]

    omega, z = phonon_modes(qpts, mat)
    Zq = mode_factors(omega, z, mat.mass_amu, params.omega_cut_eV)
    nB = bose_einstein(omega, T)
    alive = omega >= params.omega_cut_eV
    adaptive = getattr(params, "smearing", 0) == 1
    if adaptive:   # hbar v of every band at every fine-grid point (k and k+q)
        v_F = group_velocities(grid_points(F), mat, U_F)
    Lq = polar_long_range(qpts, mat, polar, Zq) if polar is not None else None

    raw = np.zeros(len(ks))
    for ik in np.unique(ks):
        sel = np.nonzero(ks == ik)[0]
        bands = bs[sel]
        k = kpts[ik]
        U_k = U_F[k_to_F[ik]]
        kq = grid_index(k[None, :] + qpts, F)
        eps_kq, U_kq = eps_F[kq], U_F[kq]
        f_kq = fermi_dirac(eps_kq, mu, T)
        if direct:
            GW = coupling_wannier_direct(np.repeat(k[None, :], Nq, axis=0), qpts, mat)
            g = bloch_coupling(GW, U_kq, np.repeat(U_k[None], Nq, axis=0)[:, :, bands], Zq)
        else:
            G = coupling_stage2(coupling_stage1(k, mat, U_k[:, bands]), qpts, mat)  # (Nq, m, b, s)
            g = rotate_final(G, U_kq, Zq)                                           # (Nq, m', b, nu)
        if Lq is not None:   # + g^L = L_q [U_{k+q}^dagger U_k]_{m' b}
            O = np.einsum("qmp,mb->qpb", np.conj(U_kq), U_k[:, bands])
            g = g + O[:, :, :, None] * Lq[:, None, None, :]
        g2 = np.abs(g) ** 2
        for jb, (j, b) in enumerate(zip(sel, bands)):
            e = eps_grid[ik, b]
            x_em = e - omega[:, None, :] - eps_kq[:, :, None]            # (Nq, m', nu)
            x_ab = e + omega[:, None, :] - eps_kq[:, :, None]
            if adaptive:   # one width per (k b, k+q m') pair, the same for every mode
                sg = adaptive_sigma(v_F[k_to_F[ik], b][None, None, :], v_F[kq], mat.lattice, nq,
                                    params.sigma_min_eV)[:, :, None]
                w = ((nB[:, None, :] + 1.0 - f_kq[:, :, None]) * gaussian_delta(x_em, sg, cut)
                     + (nB[:, None, :] + f_kq[:, :, None]) * gaussian_delta(x_ab, sg, cut))
            else:
                w = ((nB[:, None, :] + 1.0 - f_kq[:, :, None]) * gaussian_delta(x_em, sigma, cut)
                     + (nB[:, None, :] + f_kq[:, :, None]) * gaussian_delta(x_ab, sigma, cut))
            w = np.where(alive[:, None, :] & _final_ok(eps_kq, params)[:, :, None], w, 0.0)
            raw[j] = 2.0 * np.pi / Nq * np.sum(g2[:, :, jb, :] * w)

    out = raw.copy()
    for ik in np.unique(ks):
        sel = np.nonzero(ks == ik)[0]
        e = eps_grid[ik, bs[sel]]
        for a, j in enumerate(sel):
            grp = sel[np.abs(e - e[a]) < params.degen_tol_eV]
            out[j] = raw[grp].mean()
    if return_raw:
        return ks, bs, out, raw
    return ks, bs, out


def contributions(mat, params, k_indices=None, q_indices=None, table=None):
    """Per-q terms of Eq. 29: c_nk(q) with Gamma_nk(before degenerate averaging) = (1/N_q) sum_q c_nk(q).

    c_nk(q) = 2 pi sum_{m' nu} |g_{m' n nu}(k,q)|^2
              [ (n_q nu + 1 - f_{m',k+q}) delta(eps_nk - hbar w_q nu - eps_{m',k+q})
              + (n_q nu + f_{m',k+q})     delta(eps_nk + hbar w_q nu - eps_{m',k+q}) ]
    (Sec. 4.2 Eq. 29, Sec. 4.7 Eq. 61), with the readings of ``linewidths_rta``.
    These are the per-q weights an importance sampler over q needs: both the
    training targets of a learned proposal and the samples of its estimate.

    ``q_indices``: None (every q of the grid, result (n_states, N_q)) or an
    integer array (n_states, S) of q-grid indices per state (result (n_states, S)).
    Returns (k_index, band, c).
    """
    nk = tuple(int(x) for x in params.nk)
    nq = tuple(int(x) for x in params.nq)
    qpts = grid_points(nq)
    kpts = grid_points(nk)
    T, mu, sigma = params.T_K, params.mu_eV, params.sigma_eV
    cut = params.delta_cut_sigmas
    F, eps_F, U_F, k_to_F = table if table is not None else electron_table(mat, params)
    eps_grid = eps_F[k_to_F]
    ks, bs = _active(eps_grid, params)
    if k_indices is not None:
        keep = np.isin(ks, np.asarray(k_indices))
        ks, bs = ks[keep], bs[keep]
    omega, z = phonon_modes(qpts, mat)
    Zq = mode_factors(omega, z, mat.mass_amu, params.omega_cut_eV)
    nB = bose_einstein(omega, T)
    alive = omega >= params.omega_cut_eV
    width = len(qpts) if q_indices is None else np.asarray(q_indices).shape[1]
    out = np.zeros((len(ks), width))
    for j, (ik, b) in enumerate(zip(ks, bs)):
        qi = np.arange(len(qpts)) if q_indices is None else np.asarray(q_indices[j], dtype=np.int64)
        k = kpts[ik]
        U_k = U_F[k_to_F[ik]]
        kq = grid_index(k[None, :] + qpts[qi], F)
        eps_kq, U_kq = eps_F[kq], U_F[kq]
        f_kq = fermi_dirac(eps_kq, mu, T)
        G = coupling_stage2(coupling_stage1(k, mat, U_k[:, [b]]), qpts[qi], mat)   # (S, m, 1, s)
        g2 = np.abs(rotate_final(G, U_kq, Zq[qi]))[:, :, 0, :] ** 2                # (S, m', nu)
        e = eps_grid[ik, b]
        om, nb_ = omega[qi][:, None, :], nB[qi][:, None, :]
        w = ((nb_ + 1.0 - f_kq[:, :, None]) * gaussian_delta(e - om - eps_kq[:, :, None], sigma, cut)
             + (nb_ + f_kq[:, :, None]) * gaussian_delta(e + om - eps_kq[:, :, None], sigma, cut))
        w = np.where(alive[qi][:, None, :] & _final_ok(eps_kq, params)[:, :, None], w, 0.0)
        out[j] = 2.0 * np.pi * np.sum(g2 * w, axis=(1, 2))
    return ks, bs, out


def phonon_rates_elph(mat, params, table=None):
    """Phonon-electron scattering rates P^{el-ph}_{q nu} on the q grid (Sec. 4.3, the diagonal
    phonon-electron term of the phonon scattering matrix):

    P_{q nu} = -(2 pi / N_k) n_{q nu} (n_{q nu} + 1)
               sum_{k b b'} |g_{b' b nu}(k,q)|^2 (f_{k b} - f_{k+q b'}) delta(eps_{k b} - eps_{k+q b'} - hbar w_{q nu})

    with the paper's replacement f_{kb} - f_{k+q b'} -> (df/d eps)(eps_{kb}) hbar w_{q nu}, so that
    P_{q nu} = (2 pi / N_k) n (n + 1) hbar w sum_{k b b'} |g|^2 [f (1 - f) / k_B T]_{k b} delta(...).

    Readings: hbar = 1 energy units (P in eV, like Gamma); b runs over the active initial
    states of the window (the states the linewidth path sums over; outside the window
    f(1-f)/k_B T is negligible), b' over all bands at k+q; delta is the truncated Gaussian of
    Eq. 61; dead modes (hbar w < omega_cut) give 0; P is averaged over modes degenerate within
    degen_tol at the same q (the mode basis inside a degenerate subspace is arbitrary).
    Returns P with shape (N_q, 3 N_at), q in grid order.
    """
    nk = tuple(int(x) for x in params.nk)
    nq = tuple(int(x) for x in params.nq)
    qpts = grid_points(nq)
    kpts = grid_points(nk)
    Nk = len(kpts)
    T, mu, sigma = params.T_K, params.mu_eV, params.sigma_eV
    cut = params.delta_cut_sigmas
    kT = KB_EV * T
    F, eps_F, U_F, k_to_F = table if table is not None else electron_table(mat, params)
    eps_grid = eps_F[k_to_F]
    ks, bs = _active(eps_grid, params)
    omega, z = phonon_modes(qpts, mat)
    Zq = mode_factors(omega, z, mat.mass_amu, params.omega_cut_eV)
    nB = bose_einstein(omega, T)
    alive = omega >= params.omega_cut_eV
    acc = np.zeros(omega.shape)
    for ik in np.unique(ks):
        sel = np.nonzero(ks == ik)[0]
        bands = bs[sel]
        k = kpts[ik]
        U_k = U_F[k_to_F[ik]]
        kq = grid_index(k[None, :] + qpts, F)
        eps_kq, U_kq = eps_F[kq], U_F[kq]
        G = coupling_stage2(coupling_stage1(k, mat, U_k[:, bands]), qpts, mat)  # (Nq, m, b, s)
        g2 = np.abs(rotate_final(G, U_kq, Zq)) ** 2                              # (Nq, m', b, nu)
        for jb, b in enumerate(bands):
            e = eps_grid[ik, b]
            f = fermi_dirac(np.array([e]), mu, T)[0]
            d = gaussian_delta(e - eps_kq[:, :, None] - omega[:, None, :], sigma, cut)  # (Nq, m', nu)
            d = np.where(_final_ok(eps_kq, params)[:, :, None], d, 0.0)
            acc += f * (1.0 - f) / kT * np.sum(g2[:, :, jb, :] * d, axis=1)
    P = np.where(alive, 2.0 * np.pi / Nk * nB * (nB + 1.0) * omega * acc, 0.0)
    out = P.copy()
    for iq in range(len(qpts)):
        for nu in range(omega.shape[1]):
            grp = np.abs(omega[iq] - omega[iq, nu]) < params.degen_tol_eV
            out[iq, nu] = P[iq, grp].mean()
    return out


# ---------------------------------------------------- three-phonon coupling (Sec. 3.1, Sec. 4.3)

def v3_coupling(q, qp, qpp, mat, anh, omega_cut: float = 1e-4) -> np.ndarray:
    """V3(q nu, q' nu', q'' nu'') for explicit triples (Sec. 3.1, Eq. 3PhCouplingInterpolation):

    V3 = sum_{R R'} sum_{a b c} sum_{s s' s''} w e^{-i (q.R + q'.R')} V3(s a R, s' b R', s'' c 0)
         conj(Z_q[s a, nu]) conj(Z_q'[s' b, nu']) conj(Z_q''[s'' c, nu'']),

    Z the mode factors of Eq. 7 (eigenvector times sqrt(hbar^2 / (2 M_s hbar w))).  Readings: the
    printed sqrt(m m m / (w w w)) with (2/hbar)^{3/2} is read as these mode factors (masses in
    the denominator, as Eq. 7 has them; the printed form would make V3 grow with the masses);
    1/N0^3 is folded into the input; dead modes give 0.  q, qp, qpp: (n, 3) crystal coordinates.
    Returns (n, 3na, 3na, 3na) complex, eV.
    """
    q, qp, qpp = (np.atleast_2d(x) for x in (q, qp, qpp))
    Zs = []
    for x in (q, qp, qpp):
        om, z = phonon_modes(x, mat)
        Zs.append(mode_factors(om, z, mat.mass_amu, omega_cut))
    ph = np.exp(-2j * np.pi * (q @ anh.R.T.astype(np.float64) + qp @ anh.Rp.T.astype(np.float64)))  # (n, pairs)
    T = np.einsum("np,p,pabc->nabc", ph, anh.w, anh.Phi3)
    return np.einsum("nabc,nai,nbj,nck->nijk", T, np.conj(Zs[0]), np.conj(Zs[1]), np.conj(Zs[2]))


def three_phonon_diag(mat, anh, params, q_indices=None) -> np.ndarray:
    """Three-phonon part of the diagonal of the phonon scattering matrix A (Sec. 4.3):

    A_{q nu} = sum_{q' nu' nu''} [ P^{q'' nu''}_{q nu, q' nu'} + P^{q' nu', q'' nu''}_{q nu} / 2 ]
             = (2 pi / N_q) sum_{q~ nu' nu''} |W|^2 [ n n' (n''+1) d(w + w' - w'')
                                                   + (1/2) n (n'+1)(n''+1) d(w - w' - w'') ],

    W = V3(q nu, q~ nu', -q'' nu'') with q'' = q + q~ on the grid (the Kronecker delta of the
    sum over G): the coalescence partner is q' = q~, the decay partner q' = -q~, and both use
    |V3(q, q~, -(q + q~))|^2 (w', n' are even in q').  Readings: hbar = 1 energy units (A in
    eV); delta the truncated Gaussian of Eq. 61 with the fixed sigma; modes dead at any of
    the three wavevectors contribute nothing; A averaged over modes degenerate within
    degen_tol at the same q.  Returns (len(q_indices) or N_q, 3na).
    """
    nq = tuple(int(x) for x in params.nq)
    qpts = grid_points(nq)
    Nq = len(qpts)
    omega, z = phonon_modes(qpts, mat)
    Zq = mode_factors(omega, z, mat.mass_amu, params.omega_cut_eV)
    nB = bose_einstein(omega, params.T_K)
    alive = omega >= params.omega_cut_eV
    sigma, cut = params.sigma_eV, params.delta_cut_sigmas
    Rps = sorted({tuple(r) for r in anh.Rp})
    rp_index = {r: i for i, r in enumerate(Rps)}
    rp_of_pair = np.array([rp_index[tuple(r)] for r in anh.Rp])
    Rp_arr = np.array(Rps, dtype=np.float64)
    ph2 = np.exp(-2j * np.pi * (qpts @ Rp_arr.T))                   # (N_q~, R') = e^{-i q~.R'}
    grid = np.indices(nq).reshape(3, -1).T
    qi_list = np.arange(Nq) if q_indices is None else np.asarray(q_indices)
    out = np.zeros((len(qi_list), omega.shape[1]))
    for row, iq in enumerate(qi_list):
        # stage 1 at fixed q: A[R'][nu][s'b][s''c] = sum_{R} w e^{-i q.R} sum_{s a} Phi3 conj(Z_q[s a, nu])
        ph1 = anh.w * np.exp(-2j * np.pi * (anh.R.astype(np.float64) @ qpts[iq]))
        A = np.zeros((len(Rps),) + (omega.shape[1],) * 3, dtype=np.complex128)
        np.add.at(A, rp_of_pair, np.einsum("p,pabc,an->pnbc", ph1, anh.Phi3, np.conj(Zq[iq])))
        # stage 2 over q~: B[q~][nu][s'b][s''c] = sum_R' e^{-i q~.R'} A[R']
        B = np.einsum("tr,rnbc->tnbc", ph2, A)
        j = grid[iq]
        jq2 = (j[None, :] + grid) % np.array(nq)                       # q'' = q + q~
        i2 = (jq2[:, 0] * nq[1] + jq2[:, 1]) * nq[2] + jq2[:, 2]
        jm = (-jq2) % np.array(nq)                                     # -q''
        im = (jm[:, 0] * nq[1] + jm[:, 1]) * nq[2] + jm[:, 2]
        W = np.einsum("tnbc,tbi,tck->tnik", B, np.conj(Zq), np.conj(Zq[im]))
        w0 = omega[iq][None, :, None, None]
        w1 = omega[:, None, :, None]
        w2 = omega[i2][:, None, None, :]
        n0, n1, n2 = nB[iq][None, :, None, None], nB[:, None, :, None], nB[i2][:, None, None, :]
        ok = alive[iq][None, :, None, None] & alive[:, None, :, None] & alive[i2][:, None, None, :] & alive[im][:, None, None, :]
        n1s, n2s = np.where(ok, n1, 0.0), np.where(ok, n2, 0.0)
        wt = (n0 * n1s * (n2s + 1.0) * gaussian_delta(w0 + w1 - w2, sigma, cut)
              + 0.5 * n0 * (n1s + 1.0) * (n2s + 1.0) * gaussian_delta(w0 - w1 - w2, sigma, cut))
        wt = np.where(ok, wt, 0.0)
        out[row] = 2.0 * np.pi / Nq * np.sum(np.abs(W) ** 2 * wt, axis=(0, 2, 3))
    res = out.copy()
    for row, iq in enumerate(qi_list):
        for nu in range(omega.shape[1]):
            grp = np.abs(omega[iq] - omega[iq, nu]) < params.degen_tol_eV
            res[row, nu] = out[row, grp].mean()
    return res


# ------------------------------------------------- RTA transport from the linewidths (Sec. 4.2, 4.3.2)

HBAR_EV_S = 6.582119569e-16     # hbar in eV s
E_CHARGE = 1.602176634e-19      # elementary charge, C


def group_velocities(k: np.ndarray, mat, U: np.ndarray) -> np.ndarray:
    """hbar v_kb in eV A, Cartesian: the derivative of Eq. 10 with respect to k (Sec. 3.3).

    Diagonal elements of U^dagger dH/dk U with dH/dk_cart = sum_R w_R i R_cart e^{ik.R} H(R)
    (Hellmann-Feynman; the velocity of non-degenerate bands; U (nk, nw, nw) columns = bands).
    """
    k = np.atleast_2d(k)
    P = phases(k, mat.R_H) * mat.w_H[None, :]
    Rc = np.asarray(mat.R_H, dtype=np.float64) @ np.asarray(mat.lattice, dtype=np.float64)
    Hf = mat.H.reshape(len(mat.R_H), -1)
    out = np.zeros((len(k), mat.nw, 3))
    for a in range(3):
        dH = ((P * (1j * Rc[:, a])[None, :]) @ Hf).reshape(len(k), mat.nw, mat.nw)
        out[:, :, a] = np.real(np.einsum("kmb,kmn,knb->kb", np.conj(U), dH, U))
    return out


def transport_rta(mat, params, gamma: np.ndarray, ks: np.ndarray, bs: np.ndarray, table=None) -> dict:
    """Electrical conductivity, Seebeck coefficient and electronic thermal conductivity in the
    relaxation-time approximation (Sec. 4.3.2) from the linewidths of the active states.

    tau = hbar / Gamma; delta f = -tau v.(e E) df/de for a field and -tau v.grad T df/dT for a
    gradient (Sec. 4.2 with the scattering matrix reduced to its diagonal), inserted in the charge
    and energy fluxes J, Q of Sec. 4.2:
        L_n[a][b] = 1/(N_k V) sum_kb tau v_a v_b (eps - mu)^n (-df/deps),
        sigma = e^2 L_0,  S = -(1/(e T)) L_0^{-1} L_1 (electron charge -e),
        kappa_el = (1/T) (L_2 - L_1 L_0^{-1} L_1).
    Readings: no spin factor (as in Eq. 29 and the fluxes of Sec. 4.2); states with Gamma = 0
    (no scattering partner) are left out; sums over the active states of the window only.
    Returns SI values: sigma in S/m, seebeck in V/K, kappa in W/(m K) (3x3 each).
    """
    F, eps_F, U_F, k_to_F = table if table is not None else electron_table(mat, params)
    nk = tuple(int(x) for x in params.nk)
    kpts = grid_points(nk)
    f_idx = k_to_F[np.asarray(ks)]
    v = group_velocities(kpts[np.asarray(ks)], mat, U_F[f_idx])[np.arange(len(ks)), np.asarray(bs)]  # eV A
    eps = eps_F[f_idx, np.asarray(bs)]
    kT = KB_EV * params.T_K
    f = fermi_dirac(eps, params.mu_eV, params.T_K)
    mdf = f * (1.0 - f) / kT                                   # -df/deps, 1/eV
    keep = np.asarray(gamma) > 0
    tau = np.where(keep, HBAR_EV_S / np.where(keep, gamma, 1.0), 0.0)   # s
    vs = v * (E_CHARGE * 1e-10) / (HBAR_EV_S * E_CHARGE)       # m/s: (eV A) / hbar
    vol = abs(np.linalg.det(np.asarray(mat.lattice, dtype=np.float64))) * 1e-30   # m^3
    Nk = int(np.prod(nk))
    de = (eps - params.mu_eV) * E_CHARGE                       # J
    w = tau * mdf / E_CHARGE                                   # s / J
    L = [np.einsum("s,sa,sb->ab", w * de ** n, vs, vs) / (Nk * vol) for n in range(3)]
    T = params.T_K
    sigma = E_CHARGE ** 2 * L[0]
    L0i = np.linalg.inv(L[0])
    seebeck = -(1.0 / (E_CHARGE * T)) * (L0i @ L[1])
    kappa = (L[2] - L[1] @ L0i @ L[1]) / T
    return {"sigma": sigma, "seebeck": seebeck, "kappa": kappa, "L": L}
