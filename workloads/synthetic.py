"""Seeded synthetic inputs for the el-ph linewidth path.

This module only *constructs inputs*: real-space Hamiltonians H(R), harmonic
force constants Phi(R), Wannier-space couplings g(R_e, R_p) and the run
parameters.  It holds none of the method's arithmetic (no Fourier sums, no
diagonalisation, no coupling rotation, no delta accumulation), so both the
CPU oracle and the GPU library can be fed from it without sharing any step of
the computation.

The paper's own workload is GaN from DFT + Wannier90 (Sec. 6.1), which is not
available here; these instances stand in for it with the shapes of the
published method: complex H(R) and g(R_e, R_p) on Wigner-Seitz R sets that
decay with |R|, spring-model force constants that obey the acoustic sum rule,
Gamma-centred Monkhorst-Pack grids (Sec. 5.1).

Units: energies eV, lengths Angstrom, masses amu, Phi eV/A^2, g(R_e,R_p) eV/A.
Complex entries are (N(0,1) + i N(0,1))/sqrt(2) before scaling, drawn from
numpy's ``default_rng(seed)`` in the order documented per generator.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field, replace

import numpy as np

__all__ = [
    "Material",
    "RTAParams",
    "toy",
    "si_like",
    "tb_einstein",
    "wigner_seitz_set",
    "batch_material",
    "grid_fractions",
    "Anharmonic",
    "three_phonon_si_like",
    "einstein3",
]


@dataclass
class Material:
    """One crystal's real-space inputs (the arrays the C ABI ``set_*`` calls take)."""

    name: str
    nw: int                      # Wannier functions
    na: int                      # atoms in the primitive cell (3*na modes)
    mass_amu: np.ndarray         # (na,)
    lattice: np.ndarray          # (3,3) rows = primitive vectors, Angstrom
    positions: np.ndarray        # (na,3) Cartesian, Angstrom
    R_H: np.ndarray              # (nRH,3) int32 lattice coordinates
    w_H: np.ndarray              # (nRH,)  weights
    H: np.ndarray                # (nRH,nw,nw) complex128: H(R)[n][m] = <0n|H|Rm>
    R_fc: np.ndarray             # (nRf,3) int32
    w_fc: np.ndarray             # (nRf,)
    Phi: np.ndarray              # (nRf,3na,3na) float64, index (kappa*3+alpha, kappa'*3+beta)
    Re: np.ndarray               # (nRe,3) int32
    we: np.ndarray               # (nRe,)
    Rp: np.ndarray               # (nRp,3) int32
    wp: np.ndarray               # (nRp,)
    g: np.ndarray                # (nRe,nRp,nw,nw,3na) complex128; [m] = k+q side, [n] = k side

    @property
    def nmodes(self) -> int:
        return 3 * self.na


@dataclass
class RTAParams:
    """Run parameters of one linewidth calculation (mirrors ``phoebe_gpu_rta_params``)."""

    nk: tuple = (8, 8, 8)
    nq: tuple = (8, 8, 8)
    T_K: float = 300.0
    mu_eV: float = 0.0
    sigma_eV: float = 0.05
    window_eV: float = 0.0       # <= 0: every state is active
    delta_cut_sigmas: float = 6.0
    omega_cut_eV: float = 1e-4
    degen_tol_eV: float = 1e-6
    precision: int = 0           # 0 FP64, 1 split BF16, 2 split TF32, 3 BF16, 4 TF32
    k_subset: np.ndarray | None = None   # optional k-grid indices of initial states
    sampler: int = 0             # 0 full q sum, 1 learned proposal, 2 uniform proposal (importance sampling)
    sample_fraction: float = 0.05
    mix_alpha: float = 0.1
    seed: int = 0
    sampler_fp32_network: int = 0
    population_delta: float = 0.0   # > 0: population window f(1-f) > delta on initial states
    smearing: int = 0               # 0 fixed Gaussian width sigma_eV, 1 adaptive width per pair of states
    sigma_min_eV: float = 1e-3      # adaptive smearing: floor of the width
    window_final: int = 0           # 1: final states (k+q, m') also pass the window

    def with_(self, **kw) -> "RTAParams":
        return replace(self, **kw)


def grid_fractions(n) -> np.ndarray:
    """Gamma-centred grid points in crystal coordinates, index (i1*N2+i2)*N3+i3 (z fastest)."""
    n1, n2, n3 = (int(x) for x in n)
    i = np.indices((n1, n2, n3)).reshape(3, -1).T.astype(np.float64)
    return i / np.array([n1, n2, n3], dtype=np.float64)


def _cnormal(rng: np.random.Generator, shape) -> np.ndarray:
    x = rng.standard_normal(tuple(shape) + (2,))
    z = x.view(np.complex128)[..., 0]
    z *= 1.0 / np.sqrt(2.0)
    return z


def _index_of(R: np.ndarray) -> dict:
    return {tuple(int(v) for v in r): i for i, r in enumerate(R)}


def _minus_index(R: np.ndarray) -> np.ndarray:
    idx = _index_of(R)
    out = np.empty(len(R), dtype=np.int64)
    for i, r in enumerate(R):
        key = tuple(int(-v) for v in r)
        if key not in idx:
            raise ValueError("R set is not closed under -R")
        out[i] = idx[key]
    return out


def _hermitian_pair_sym(X: np.ndarray, minus: np.ndarray) -> np.ndarray:
    """H(R) = (X(R) + X(-R)^dagger)/2 so that H(-R) = H(R)^dagger."""
    return 0.5 * (X + np.conj(np.swapaxes(X[minus], -1, -2)))


def _coupling_sym(X: np.ndarray, minus_e: np.ndarray, minus_p: np.ndarray) -> np.ndarray:
    """g[m][n][ka](Re,Rp) = (X[m][n][ka](Re,Rp) + conj X[n][m][ka](-Re,-Rp))/2, in place-ish."""
    out = np.empty_like(X)
    for ie in range(X.shape[0]):
        Y = X[minus_e[ie]][minus_p]            # (nRp, nw, nw, nmodes)
        out[ie] = 0.5 * (X[ie] + np.conj(np.swapaxes(Y, 1, 2)))
    return out


def wigner_seitz_set(lattice: np.ndarray, n_super: int, rmax: float | None = None):
    """Lattice vectors of the Wigner-Seitz cell of the n_super^3 supercell.

    Returns (R int32 (n,3), weights = 1/degeneracy).  With ``rmax`` the set is
    truncated to |R| <= rmax (whole shells), which keeps it closed under -R.
    """
    N = int(n_super)
    rng_ = range(-2 * N, 2 * N + 1)
    pts = np.array(list(itertools.product(rng_, rng_, rng_)), dtype=np.int64)
    T = np.array(list(itertools.product(range(-2, 3), repeat=3)), dtype=np.int64) * N
    cart = pts @ lattice
    d0 = np.linalg.norm(cart, axis=1)
    keepR, keepW = [], []
    Tc = T @ lattice
    for i in np.argsort(d0, kind="stable"):
        ds = np.linalg.norm(cart[i][None, :] + Tc, axis=1)
        dmin = ds.min()
        if d0[i] <= dmin + 1e-8:
            deg = int(np.sum(np.abs(ds - dmin) < 1e-8))
            keepR.append(pts[i])
            keepW.append(1.0 / deg)
    R = np.array(keepR, dtype=np.int64)
    w = np.array(keepW, dtype=np.float64)
    if rmax is not None:
        L = np.linalg.norm(R @ lattice, axis=1)
        sel = L <= rmax + 1e-9
        R, w = R[sel], w[sel]
    # deterministic order: by length, then lexicographic
    L = np.linalg.norm(R @ lattice, axis=1)
    order = np.lexsort((R[:, 2], R[:, 1], R[:, 0], np.round(L, 9)))
    return R[order].astype(np.int32), w[order]


def _central_springs(lattice, positions, springs, search=3):
    """Harmonic force constants of central springs, acoustic sum rule on the self term.

    ``springs`` = list of (bond length, k eV/A^2).  For a bond d between atom
    kappa (cell 0) and kappa' (cell R): Phi[k a, k' b](R) -= k d_a d_b / |d|^2
    and Phi[k a, k b](0) += k d_a d_b / |d|^2.
    """
    na = len(positions)
    rng_ = range(-search, search + 1)
    terms = {}
    def add(R, i, j, blk):
        key = tuple(int(v) for v in R)
        if key not in terms:
            terms[key] = np.zeros((3 * na, 3 * na))
        terms[key][3 * i:3 * i + 3, 3 * j:3 * j + 3] += blk
    for R in itertools.product(rng_, rng_, rng_):
        Rc = np.array(R, dtype=np.float64) @ lattice
        for i in range(na):
            for j in range(na):
                d = Rc + positions[j] - positions[i]
                L = np.linalg.norm(d)
                if L < 1e-9:
                    continue
                for (blen, kspr) in springs:
                    if abs(L - blen) < 1e-6 * max(1.0, blen):
                        u = d / L
                        blk = kspr * np.outer(u, u)
                        add(R, i, j, -blk)
                        add((0, 0, 0), i, i, blk)
    keys = sorted(terms.keys(), key=lambda r: (sum(v * v for v in r), r))
    R = np.array(keys, dtype=np.int32)
    Phi = np.array([terms[k] for k in keys])
    return R, np.ones(len(R)), Phi


def toy(seed: int = 0) -> tuple[Material, RTAParams]:
    """Simple-cubic toy: 2 Wannier functions, 1 atom (28 amu), R sets {-1,0,1}^3.

    Draw order: H's X(R) (27,2,2) complex, then g's X (27,27,2,2,3) complex.
    H(R) = sym(X(R) e^{-|R|/0.7}); g = sym(X e^{-(|Re|+|Rp|)/0.7}) (Hermitian pair
    symmetrisation); Phi from nearest-neighbour central springs k = 1 eV/A^2.
    Grids 8^3 x 8^3, T = 300 K, mu = tr H(0)/2, sigma = 0.05 eV, no window.
    """
    rng = np.random.default_rng(seed)
    lat = np.eye(3)
    R = np.array(list(itertools.product((-1, 0, 1), repeat=3)), dtype=np.int32)
    L = np.linalg.norm(R.astype(float), axis=1)
    minus = _minus_index(R)
    nw, na = 2, 1
    XH = _cnormal(rng, (len(R), nw, nw)) * np.exp(-L / 0.7)[:, None, None]
    H = _hermitian_pair_sym(XH, minus)
    Xg = _cnormal(rng, (len(R), len(R), nw, nw, 3 * na))
    Xg *= np.exp(-(L[:, None] + L[None, :]) / 0.7)[:, :, None, None, None]
    g = _coupling_sym(Xg, minus, minus)
    Rf, wf, Phi = _central_springs(lat, np.zeros((1, 3)), [(1.0, 1.0)], search=1)
    mat = Material("toy", nw, na, np.array([28.0]), lat, np.zeros((1, 3)),
                   R, np.ones(len(R)), H, Rf, wf, Phi,
                   R.copy(), np.ones(len(R)), R.copy(), np.ones(len(R)), g)
    mu = float(np.real(np.trace(H[_index_of(R)[(0, 0, 0)]])) / nw)
    return mat, RTAParams(nk=(8, 8, 8), nq=(8, 8, 8), T_K=300.0, mu_eV=mu,
                          sigma_eV=0.05, window_eV=0.0)


SI_A = 5.431


def si_like(seed: int = 0, nk: int = 40, nq: int | None = None,
            nw: int = 8) -> tuple[Material, RTAParams]:
    """fcc Si-like crystal: 8 Wannier functions, 2 atoms (28.0855 amu), 429 R vectors.

    R set: Wigner-Seitz set of the 8^3 supercell (617 vectors) cut to whole
    shells |R| <= 2.9155 a (429 vectors, weights 1), shared by H, R_e and R_p.
    Decay length l = 0.7 a/sqrt(2).  Draw order: H's X (429,nw,nw), then g's X
    (429,429,nw,nw,6).  Phi: nearest-neighbour (sqrt(3)a/4) springs 10 eV/A^2
    plus next-nearest (a/sqrt(2)) springs 2 eV/A^2.
    Grids nk^3 x nq^3 (default 40^3), T = 300 K, sigma = 0.02 eV,
    window +-0.5 eV around mu = tr H(0)/nw.
    """
    a = SI_A
    lat = 0.5 * a * np.array([[0, 1, 1], [1, 0, 1], [1, 1, 0]], dtype=np.float64)
    pos = np.array([[0, 0, 0], [0.25 * a, 0.25 * a, 0.25 * a]])
    R, w = wigner_seitz_set(lat, 8, rmax=2.9155 * a)
    w = np.ones(len(R))
    L = np.linalg.norm(R @ lat, axis=1)
    ell = 0.7 * a / np.sqrt(2.0)
    minus = _minus_index(R)
    rng = np.random.default_rng(seed)
    na = 2
    XH = _cnormal(rng, (len(R), nw, nw)) * np.exp(-L / ell)[:, None, None]
    H = _hermitian_pair_sym(XH, minus)
    Xg = _cnormal(rng, (len(R), len(R), nw, nw, 3 * na))
    decay = np.exp(-(L[:, None] + L[None, :]) / ell)
    Xg *= decay[:, :, None, None, None]
    g = _coupling_sym(Xg, minus, minus)
    del Xg
    Rf, wf, Phi = _central_springs(lat, pos, [(np.sqrt(3.0) * a / 4.0, 10.0),
                                              (a / np.sqrt(2.0), 2.0)], search=2)
    mat = Material("si_like", nw, na, np.array([28.0855, 28.0855]), lat, pos,
                   R, w, H, Rf, wf, Phi, R.copy(), w.copy(), R.copy(), w.copy(), g)
    mu = float(np.real(np.trace(H[_index_of(R)[(0, 0, 0)]])) / nw)
    nqv = nk if nq is None else nq
    return mat, RTAParams(nk=(nk, nk, nk), nq=(nqv, nqv, nqv), T_K=300.0, mu_eV=mu,
                          sigma_eV=0.02, window_eV=0.5)


def tb_einstein(eps0: float = 0.0, t: float = 0.25, lam: float = 0.215,
                c=(0.3, -0.2, 0.1), mass: float = 28.0, n: int = 8,
                sigma: float = 0.05, T_K: float = 300.0, mu: float = 0.1,
                hop_phase: float = 0.0) -> tuple[Material, RTAParams]:
    """Closed-form case: one band, one atom, Einstein phonon, constant coupling.

    H(0) = eps0, H(+-x,+-y,+-z) = -t e^{+-i hop_phase}, so that
    eps(k) = eps0 - 2t sum_a cos(2 pi k_a + hop_phase).  Phi(0) = M lam I, so the
    mass-scaled dynamical matrix is lam*I at every q (one Einstein frequency,
    lam in eV/(A^2 amu)).  g(Re=0,Rp=0)[0][0][a] = c_a.  No randomness.
    """
    lat = np.eye(3)
    hops = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    R = np.array(hops, dtype=np.int32)
    H = np.zeros((len(R), 1, 1), dtype=np.complex128)
    H[0, 0, 0] = eps0
    for i, r in enumerate(hops[1:], start=1):
        s = 1.0 if sum(r) > 0 else -1.0
        H[i, 0, 0] = -t * np.exp(1j * s * hop_phase)
    Phi = (mass * lam * np.eye(3))[None, :, :]
    Rf = np.zeros((1, 3), dtype=np.int32)
    g = np.zeros((1, 1, 1, 1, 3), dtype=np.complex128)
    g[0, 0, 0, 0, :] = np.asarray(c, dtype=np.complex128)
    Z0 = np.zeros((1, 3), dtype=np.int32)
    mat = Material("tb_einstein", 1, 1, np.array([mass]), lat, np.zeros((1, 3)),
                   R, np.ones(len(R)), H, Rf, np.ones(1), Phi,
                   Z0, np.ones(1), Z0.copy(), np.ones(1), g)
    return mat, RTAParams(nk=(n, n, n), nq=(n, n, n), T_K=T_K, mu_eV=mu,
                          sigma_eV=sigma, window_eV=0.0)


def tb_einstein2(eps0: float = 0.05, t: float = 0.25, lam=(0.215, 0.6), mass=(28.0, 12.0),
                 c=(0.3, -0.2, 0.1), d=(0.1, 0.25, -0.15), n: int = 6, sigma: float = 0.05,
                 T_K: float = 300.0, mu: float = 0.1) -> tuple[Material, RTAParams]:
    """One band, two atoms with independent Einstein springs (two frequencies), constant coupling.

    The band is that of ``tb_einstein``; Phi(0) = diag(M1 lam1 I, M2 lam2 I), so the modes are
    hbar w_s = 0.06465 sqrt(lam_s), three per atom, their eigenvectors on one atom each;
    g(Re=0,Rp=0)[0][0][3s + a] = c_a (s = 0) or d_a (s = 1).  No randomness.
    """
    mat1, prm = tb_einstein(eps0=eps0, t=t, lam=lam[0], c=c, mass=mass[0], n=n, sigma=sigma, T_K=T_K, mu=mu)
    Phi = np.zeros((1, 6, 6))
    Phi[0, :3, :3] = mass[0] * lam[0] * np.eye(3)
    Phi[0, 3:, 3:] = mass[1] * lam[1] * np.eye(3)
    g = np.zeros((1, 1, 1, 1, 6), dtype=np.complex128)
    g[0, 0, 0, 0, :3] = np.asarray(c, dtype=np.complex128)
    g[0, 0, 0, 0, 3:] = np.asarray(d, dtype=np.complex128)
    Z0 = np.zeros((1, 3), dtype=np.int32)
    mat = Material("tb_einstein2", 1, 2, np.array(mass, dtype=np.float64), np.eye(3),
                   np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]]), mat1.R_H, mat1.w_H, mat1.H,
                   np.zeros((1, 3), dtype=np.int32), np.ones(1), Phi, Z0, np.ones(1), Z0.copy(), np.ones(1), g)
    return mat, prm


def material_of_shape(name: str, nw: int, na: int, nR_target: int, n: int, rng: np.random.Generator,
                      g_budget_bytes: float = 256e6) -> tuple[Material, RTAParams]:
    """A crystal of a given shape built by the Si-like rules (fcc lattice, decaying seeded H and g).

    H(R) and the force constants use the whole-shell cut of the fcc Wigner-Seitz set (8^3
    supercell, 617 vectors, else 12^3) nearest to nR_target vectors.  The el-ph coupling
    g(Re,Rp) uses the largest whole-shell prefix of that set whose complex128 tensor
    (nRe * nRp * nw^2 * 3na * 16 bytes) stays within g_budget_bytes (at least R = 0): a
    1200-vector set with 24 Wannier functions and 6 atoms would need 239 GB.
    Atoms sit at seeded positions in the fcc cell, >= 0.2 a apart; springs between every
    distinct bond length below 0.75 a with constants uniform in [2,12] eV/A^2.
    Grid n^3 for k and q, T = 300 K, sigma = 0.02 eV, window +-0.5 eV around mu = tr H(0)/nw.
    """
    a = SI_A
    lat = 0.5 * a * np.array([[0, 1, 1], [1, 0, 1], [1, 1, 0]], dtype=np.float64)
    nsup = 8 if nR_target <= 617 else 12
    Rall, _ = wigner_seitz_set(lat, nsup)
    Lall = np.linalg.norm(Rall @ lat, axis=1)
    Lr = np.round(Lall, 6)
    shells = np.unique(Lr)
    counts = np.array([np.sum(Lr <= s) for s in shells])
    cut = shells[int(np.argmin(np.abs(counts - nR_target)))]
    order = np.argsort(Lr, kind="stable")
    Rall, Lall, Lr = Rall[order], Lall[order], Lr[order]
    sel = Lr <= cut
    R = Rall[sel]
    L = Lall[sel]
    minus = _minus_index(R)
    per_pair = float(nw * nw * 3 * na * 16)
    g_cut = shells[0]
    for sh, cnt in zip(shells, counts):
        if sh <= cut and cnt * cnt * per_pair <= g_budget_bytes:
            g_cut = sh
    gsel = np.round(L, 6) <= g_cut
    Rg, Lg = R[gsel], L[gsel]
    minus_g = _minus_index(Rg)
    ell = 0.7 * a / np.sqrt(2.0)
    pos = [np.zeros(3)]
    while len(pos) < na:
        p = rng.uniform(0.0, 1.0, 3) @ lat
        if all(np.linalg.norm(p - q) > 0.2 * a for q in pos):
            pos.append(p)
    pos = np.array(pos)
    mass = rng.uniform(10.0, 120.0, na)
    XH = _cnormal(rng, (len(R), nw, nw)) * np.exp(-L / ell)[:, None, None]
    H = _hermitian_pair_sym(XH, minus)
    Xg = _cnormal(rng, (len(Rg), len(Rg), nw, nw, 3 * na))
    Xg *= np.exp(-(Lg[:, None] + Lg[None, :]) / ell)[:, :, None, None, None]
    g = _coupling_sym(Xg, minus_g, minus_g)
    del Xg
    bonds = set()
    for R3 in itertools.product(range(-2, 3), repeat=3):
        Rc = np.array(R3, dtype=float) @ lat
        for i in range(na):
            for j in range(na):
                d = np.linalg.norm(Rc + pos[j] - pos[i])
                if 1e-9 < d < 0.75 * a:
                    bonds.add(round(d, 6))
    springs = [(b, float(rng.uniform(2.0, 12.0))) for b in sorted(bonds)]
    Rf, wf, Phi = _central_springs(lat, pos, springs, search=2)
    w = np.ones(len(R))
    wg = np.ones(len(Rg))
    mat = Material(name, nw, na, mass, lat, pos, R.astype(np.int32), w, H,
                   Rf, wf, Phi, Rg.astype(np.int32), wg, Rg.astype(np.int32), wg.copy(), g)
    mu = float(np.real(np.trace(H[_index_of(R)[(0, 0, 0)]])) / nw)
    return mat, RTAParams(nk=(n, n, n), nq=(n, n, n), T_K=300.0, mu_eV=mu,
                          sigma_eV=0.02, window_eV=0.5)


def batch_shape(index: int, seed: int = 0) -> tuple[int, int, int, int]:
    """Shape (nw, na, nR_target, n) of material `index` of the batching workload: uniform draws
    nw in [4,24], na in [1,6], |R| in [100,1200], grid n in [16,40], seeded by (seed, index)."""
    rng = np.random.default_rng([seed, index])
    return (int(rng.integers(4, 25)), int(rng.integers(1, 7)), int(rng.integers(100, 1201)),
            int(rng.integers(16, 41)))


def batch_material(index: int, seed: int = 0, g_budget_bytes: float = 256e6) -> tuple[Material, RTAParams]:
    """One of the uneven materials of the batching workload (shape from ``batch_shape``)."""
    rng = np.random.default_rng([seed, index])
    nw, na, nR_target, n = (int(rng.integers(4, 25)), int(rng.integers(1, 7)), int(rng.integers(100, 1201)),
                            int(rng.integers(16, 41)))
    return material_of_shape(f"batch{index}", nw, na, nR_target, n, rng, g_budget_bytes)


# ------------------------------------------------------------ third-order force constants

@dataclass
class Anharmonic:
    """Third-order force constants V3(s a R, s' b R', s'' c 0) on a list of (R, R') pairs
    (the arrays the C ABI ``set_force_constants3`` takes); any 1/N0^3 is folded in."""

    R: np.ndarray                # (n,3) int32
    Rp: np.ndarray               # (n,3) int32
    w: np.ndarray                # (n,) weights
    Phi3: np.ndarray             # (n, 3na, 3na, 3na) float64, eV/A^3, [s a][s' b][s'' c]


def _phonon_only_material(name, lat, pos, masses, Rf, wf, Phi):
    """A material with phonons only: one Wannier function with H = 0 and a zero coupling
    (the three-phonon path needs the harmonic and third-order force constants alone)."""
    Z0 = np.zeros((1, 3), dtype=np.int32)
    na = len(masses)
    return Material(name, 1, na, np.asarray(masses, dtype=np.float64), lat, pos, Z0, np.ones(1),
                    np.zeros((1, 1, 1), dtype=np.complex128), Rf, wf, Phi, Z0.copy(), np.ones(1), Z0.copy(),
                    np.ones(1), np.zeros((1, 1, 1, 1, 3 * na), dtype=np.complex128))


def three_phonon_si_like(seed: int = 0, nq: int = 16, shell: float = 0.75) -> tuple[Material, Anharmonic, RTAParams]:
    """fcc Si-like crystal (two atoms, the spring model of ``si_like``) with random third-order
    force constants on the (R, R') pairs of the lattice vectors with |R| <= shell * a, decaying as
    exp(-(|R| + |R'|) / (0.4 a)), 2 eV/A^3 at R = R' = 0.  Draw order: one (n, 6, 6, 6) normal
    array.  q grid nq^3, T = 300 K, sigma = 2 meV.  Not symmetrised (the interpolation of
    Eq. 3PhCouplingInterpolation needs none)."""
    a = SI_A
    lat = 0.5 * a * np.array([[0, 1, 1], [1, 0, 1], [1, 1, 0]], dtype=np.float64)
    pos = np.array([[0, 0, 0], [0.25 * a, 0.25 * a, 0.25 * a]])
    Rf, wf, Phi = _central_springs(lat, pos, [(np.sqrt(3.0) * a / 4.0, 10.0), (a / np.sqrt(2.0), 2.0)], search=2)
    mat = _phonon_only_material("si_like_3ph", lat, pos, [28.0855, 28.0855], Rf, wf, Phi)
    S = np.array([r for r in itertools.product(range(-2, 3), repeat=3)
                  if np.linalg.norm(np.array(r) @ lat) <= shell * a + 1e-9], dtype=np.int32)
    R = np.repeat(S, len(S), axis=0)
    Rp = np.tile(S, (len(S), 1))
    L = np.linalg.norm(R @ lat, axis=1) + np.linalg.norm(Rp @ lat, axis=1)
    rng = np.random.default_rng(seed)
    Phi3 = rng.normal(size=(len(R), 6, 6, 6)) * (2.0 * np.exp(-L / (0.4 * a)))[:, None, None, None]
    anh = Anharmonic(R.astype(np.int32), Rp.astype(np.int32), np.ones(len(R)), Phi3)
    return mat, anh, RTAParams(nk=(nq, nq, nq), nq=(nq, nq, nq), T_K=300.0, sigma_eV=0.002, window_eV=0.0)


def einstein3(lam1: float = 0.1, mass1: float = 28.0, mass2: float = 20.0, n: int = 6, T_K: float = 300.0,
              sigma: float = 0.002, offsite=None, seed: int = 4) -> tuple[Material, Anharmonic, RTAParams]:
    """Closed-form case of the three-phonon path: simple cubic (a = 1 A), two atoms at the origin
    with Einstein springs, D = diag(lam1 I, 4 lam1 I) (hbar w2 = 2 hbar w1, exactly resonant for
    w2 -> w1 + w1), and third-order constants on one (R, R') pair: (0, 0), or ``offsite`` =
    (R0, R0').  Phi3 = the (6, 6, 6) normal draw of ``seed``."""
    lat = np.eye(3)
    pos = np.zeros((2, 3))
    Phi = np.zeros((1, 6, 6))
    Phi[0, :3, :3] = mass1 * lam1 * np.eye(3)
    Phi[0, 3:, 3:] = mass2 * 4.0 * lam1 * np.eye(3)
    mat = _phonon_only_material("einstein3", lat, pos, [mass1, mass2], np.zeros((1, 3), dtype=np.int32),
                                np.ones(1), Phi)
    R0, R0p = ((0, 0, 0), (0, 0, 0)) if offsite is None else offsite
    Phi3 = np.random.default_rng(seed).normal(size=(1, 6, 6, 6))
    anh = Anharmonic(np.array([R0], dtype=np.int32), np.array([R0p], dtype=np.int32), np.ones(1), Phi3)
    return mat, anh, RTAParams(nk=(n, n, n), nq=(n, n, n), T_K=T_K, sigma_eV=sigma, window_eV=0.0)
