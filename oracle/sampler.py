"""Plain FP64 CPU oracle of the learned q proposal and its importance-sampled Gamma.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library.

The paper (arXiv 2111.14999) sums Eq. 29 over every q of the grid.  This
module states the sampled alternative the library adds on top of it:

  * per active state (n, k) the q-resolved terms c_nk(q) of Eq. 29
    (``oracle.elph.contributions``), so that Gamma_nk = (1/N_q) sum_q c_nk(q);
  * a multilayer perceptron z(x) over features x = (q~, eps_nk - mu, v_nk)
    (q~: q wrapped into [-1/2, 1/2) per axis; v_nk = <n| dH/dk |n> / 2 pi with
    the Fourier derivative of Eq. 10), 7 -> 128 -> 128 -> 128 -> 1 with SiLU,
    whose parameters are rounded to BF16;
  * per state the shell factor phi_nk(q): the bracket of Eq. 29 with |g|^2
    replaced by 1/(hbar w_q nu), summed over final bands and live modes (zero
    exactly where every Gaussian of the q term is cut, so zero wherever
    c_nk(q) is);
  * per k the defensive mixture p_k(q) = (1 - a) mean_n softmax_q (z_nk(q) +
    log phi_nk(q)) + a mean_n phi_nk(q) / sum_q phi_nk, over the active bands n
    with some phi > 0 (uniform when there is none: then every c is 0);
  * S i.i.d. draws q_j from p_k (inverse CDF in q-index order, FP64, driven by
    Philox4x32-10 uniforms) and the unbiased estimate
    Gamma^_nk = (1/S) sum_j c_nk(q_j) / (N_q p_k(q_j));
  * the training loss: per state the cross entropy between the target
    distribution t(q) = c(q) / sum_q c and softmax_q (z(q) + log phi(q)),
    averaged over states;
  * the network-free alternatives: the shell proposal mean_n phi_nk / sum phi_nk
    and the uniform proposal 1/N_q.

Parameter blob (float32, the library's layout): W1[128][7], b1[128], W2[128][128],
b2[128], W3[128][128], b3[128], w4[128], b4 -- 34177 numbers.
"""
from __future__ import annotations

import numpy as np

from . import elph

NIN, NH = 7, 128
SHAPES = (("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)),
          ("W3", (NH, NH)), ("b3", (NH,)), ("w4", (NH,)), ("b4", (1,)))
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)

# Philox4x32-10 constants (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11)
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
IS_STREAM = 0x4953          # third counter word of the importance-sampling draws


# ------------------------------------------------------------------ counter-based generator

def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32 with 10 rounds: ctr (N,4) uint32, key (k0, k1) -> (N,4) uint32.

    One round maps (c0, c1, c2, c3) with key (k0, k1) to
    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)), and the key
    advances by the Weyl increments (W0, W1) between rounds.
    """
    c = np.asarray(ctr, dtype=np.uint64).reshape(-1, 4).copy()
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    mask = np.uint64(0xFFFFFFFF)
    for _ in range(10):
        p0 = c[:, 0] * np.uint64(PHILOX_M0)
        p1 = c[:, 2] * np.uint64(PHILOX_M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        c = np.stack([hi1 ^ c[:, 1] ^ np.uint64(k0), lo1, hi0 ^ c[:, 3] ^ np.uint64(k1), lo0], axis=1)
        k0 = (k0 + PHILOX_W0) & 0xFFFFFFFF
        k1 = (k1 + PHILOX_W1) & 0xFFFFFFFF
    return c.astype(np.uint32)


def is_uniforms(seed: int, k_index: int, n: int) -> np.ndarray:
    """The n uniforms in [0,1) of one k point's draws: draw j uses counter (j, k, IS_STREAM, 0),
    key (seed low word, seed high word), and u = ((x1 << 32 | x0) >> 11) * 2^-53 of the output words."""
    ctr = np.zeros((n, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(n, dtype=np.uint64)
    ctr[:, 1] = np.uint64(k_index)
    ctr[:, 2] = np.uint64(IS_STREAM)
    x = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)).astype(np.uint64)
    bits = ((x[:, 1] << np.uint64(32)) | x[:, 0]) >> np.uint64(11)
    return bits.astype(np.float64) * 2.0 ** -53


# ------------------------------------------------------------------ parameters

def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest BF16 (ties to even); returned as float64."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(blob: np.ndarray) -> dict:
    """Blob -> dict of FP64 arrays (no rounding)."""
    blob = np.asarray(blob, dtype=np.float64).ravel()
    if blob.size != NPARAM:
        raise ValueError(f"parameter blob has {blob.size} numbers, expected {NPARAM}")
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = blob[o:o + n].reshape(shape).copy()
        o += n
    return out


def pack(theta: dict) -> np.ndarray:
    return np.concatenate([np.asarray(theta[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16_params(blob: np.ndarray) -> dict:
    """The parameters the network computes with: the float32 blob rounded to BF16."""
    return unpack(bf16_round(np.asarray(blob, dtype=np.float32)))


# ------------------------------------------------------------------ network

def silu(a):
    return a / (1.0 + np.exp(-a))


def mlp_forward(theta: dict, X: np.ndarray):
    """z = w4 . h3 + b4, h_l = silu(W_l h_{l-1} + b_l), h_0 = x.  Returns (z, cache)."""
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ theta["W1"].T + theta["b1"]
    h1 = silu(a1)
    a2 = h1 @ theta["W2"].T + theta["b2"]
    h2 = silu(a2)
    a3 = h2 @ theta["W3"].T + theta["b3"]
    h3 = silu(a3)
    z = h3 @ theta["w4"] + theta["b4"][0]
    return z, (X, a1, h1, a2, h2, a3, h3)


def silu_grad(a):
    s = 1.0 / (1.0 + np.exp(-a))
    return s * (1.0 + a * (1.0 - s))


def mlp_backward(theta: dict, cache, dz: np.ndarray) -> dict:
    """Gradients of sum_r dz_r z_r with respect to every parameter (chain rule, layer by layer)."""
    X, a1, h1, a2, h2, a3, h3 = cache
    g = {"w4": h3.T @ dz, "b4": np.array([dz.sum()])}
    d3 = np.outer(dz, theta["w4"]) * silu_grad(a3)
    g["W3"], g["b3"] = d3.T @ h2, d3.sum(0)
    d2 = (d3 @ theta["W3"]) * silu_grad(a2)
    g["W2"], g["b2"] = d2.T @ h1, d2.sum(0)
    d1 = (d2 @ theta["W2"]) * silu_grad(a1)
    g["W1"], g["b1"] = d1.T @ X, d1.sum(0)
    return g


def softmax_ce(z: np.ndarray, group_off: np.ndarray, target: np.ndarray, prior: np.ndarray | None = None):
    """Loss (1/G) sum_groups -sum_{r in group} t_r log softmax(z + prior)_r with t normalised per group,
    and its gradient dL/dz = (softmax(z + prior) - t) / G.  ``prior``: per-row additive log-weights
    (-inf allowed where the target is 0), default 0."""
    G = len(group_off) - 1
    loss, dz = 0.0, np.zeros_like(z)
    for g in range(G):
        a, b = int(group_off[g]), int(group_off[g + 1])
        zz = z[a:b] + (prior[a:b] if prior is not None else 0.0)
        m = zz.max()
        lse = m + np.log(np.sum(np.exp(zz - m)))
        t = target[a:b] / np.sum(target[a:b])
        pos = t > 0
        loss += -np.sum(t[pos] * (zz[pos] - lse))
        dz[a:b] = (np.exp(zz - lse) - t) / G
    return loss / G, dz


def loss_and_grad(blob: np.ndarray, X: np.ndarray, group_off: np.ndarray, target: np.ndarray,
                  prior: np.ndarray | None = None):
    """Training loss and its gradient (as a blob) at the BF16-rounded parameters of ``blob``."""
    theta = bf16_params(blob)
    z, cache = mlp_forward(theta, X)
    loss, dz = softmax_ce(z, np.asarray(group_off), np.asarray(target, dtype=np.float64),
                          None if prior is None else np.asarray(prior, dtype=np.float64))
    return loss, pack(mlp_backward(theta, cache, dz)), z


# ------------------------------------------------------------------ features

def wrapped_q(nq) -> np.ndarray:
    """q~ = q - floor(q + 1/2) per axis, in [-1/2, 1/2), for every q of the grid (index order)."""
    q = elph.grid_points(nq)
    return q - np.floor(q + 0.5)


def band_velocities(k: np.ndarray, mat, U: np.ndarray) -> np.ndarray:
    """v[k, b, i] = Re <u_b| sum_R w_R i R_i e^{i k.R} H(R) |u_b>  = (1/2 pi) d eps_b / d k_i
    (Hellmann-Feynman on Eq. 10, k in crystal coordinates), for U (nk, nw, nw) columns = bands."""
    k = np.atleast_2d(k)
    P = elph.phases(k, mat.R_H) * mat.w_H[None, :]
    out = np.zeros((len(k), mat.nw, 3))
    Hf = mat.H.reshape(len(mat.R_H), -1)
    for i in range(3):
        dH = ((P * (1j * mat.R_H[:, i])[None, :]) @ Hf).reshape(len(k), mat.nw, mat.nw)
        out[:, :, i] = np.real(np.einsum("kmb,kmn,knb->kb", np.conj(U), dH, U))
    return out


def state_features(mat, params, ks, bs, table=None) -> np.ndarray:
    """Per state (eps_nk - mu, v_nk[0..2]), shape (n_states, 4)."""
    F, eps_F, U_F, k_to_F = table if table is not None else elph.electron_table(mat, params)
    kpts = elph.grid_points(tuple(int(x) for x in params.nk))
    f = k_to_F[np.asarray(ks)]
    v = band_velocities(kpts[np.asarray(ks)], mat, U_F[f])
    out = np.empty((len(ks), 4))
    out[:, 0] = eps_F[f, np.asarray(bs)] - params.mu_eV
    out[:, 1:] = v[np.arange(len(ks)), np.asarray(bs)]
    return out


def rows_for_state(feat: np.ndarray, qt: np.ndarray) -> np.ndarray:
    """Network inputs of one state over the q points qt (S,3): rows (q~, eps - mu, v)."""
    X = np.empty((len(qt), NIN))
    X[:, :3] = qt
    X[:, 3:] = feat[None, :]
    return X


# ------------------------------------------------------------------ shell factor

def shell_factor(mat, params, ks, bs, table=None, q_indices=None) -> np.ndarray:
    """phi_nk(q) = sum_{m'} sum_{nu: hbar w_q nu >= omega_cut} [ (n_q nu + 1 - f_m'k+q) D(eps_nk - hbar w_q nu - eps_m'k+q)
                  + (n_q nu + f_m'k+q) D(eps_nk + hbar w_q nu - eps_m'k+q) ] / (hbar w_q nu),
    D(x) = exp(-x^2 / sigma^2) for |x| < cut sigma and 0 beyond: the bracket of Eq. 29 (Sec. 4.2,
    Gaussian of Eq. 61 without its normalisation) with |g_m'n nu|^2 replaced by 1/(hbar w_q nu).
    Every term of c_nk(q) carries one of these weights, so phi_nk(q) = 0 implies c_nk(q) = 0.
    Returns (n_states, N_q) for every q of the grid (or (n_states, len(q_indices[s])))."""
    F, eps_F, U_F, k_to_F = table if table is not None else elph.electron_table(mat, params)
    nq = tuple(int(x) for x in params.nq)
    qpts = elph.grid_points(nq)
    kpts = elph.grid_points(tuple(int(x) for x in params.nk))
    omega, _ = elph.phonon_modes(qpts, mat)
    nB = elph.bose_einstein(omega, params.T_K)
    alive = omega >= params.omega_cut_eV
    inv_w = np.where(alive, 1.0 / np.where(alive, omega, 1.0), 0.0)
    sig, xcut = params.sigma_eV, params.delta_cut_sigmas * params.sigma_eV
    ks, bs = np.asarray(ks), np.asarray(bs)
    out = []
    for j, (k, b) in enumerate(zip(ks, bs)):
        qi = np.arange(len(qpts)) if q_indices is None else np.asarray(q_indices[j])
        e = eps_F[k_to_F[k], b]
        kq = elph.grid_index(kpts[k][None, :] + qpts[qi], F)
        ekq = eps_F[kq]                                              # (nq, m')
        f = elph.fermi_dirac(ekq, params.mu_eV, params.T_K)
        x1 = e - omega[qi][:, None, :] - ekq[:, :, None]             # (nq, m', nu)
        x2 = e + omega[qi][:, None, :] - ekq[:, :, None]
        d1 = np.where(np.abs(x1) < xcut, np.exp(-(x1 / sig) ** 2), 0.0)
        d2 = np.where(np.abs(x2) < xcut, np.exp(-(x2 / sig) ** 2), 0.0)
        w = (nB[qi][:, None, :] + 1.0 - f[:, :, None]) * d1 + (nB[qi][:, None, :] + f[:, :, None]) * d2
        out.append(np.sum(w * inv_w[qi][:, None, :], axis=(1, 2)))
    return np.array(out).reshape(len(ks), -1)


def log_shell(phi: np.ndarray) -> np.ndarray:
    """log phi with -inf where phi = 0."""
    phi = np.asarray(phi, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return np.where(phi > 0, np.log(np.where(phi > 0, phi, 1.0)), -np.inf)


# ------------------------------------------------------------------ importance sampling

def _softmax_rows(x: np.ndarray) -> np.ndarray:
    m = x.max(axis=1, keepdims=True)
    e = np.exp(x - m)
    return e / e.sum(axis=1, keepdims=True)


def proposal(logits: np.ndarray, alpha: float, log_phi: np.ndarray | None = None) -> np.ndarray:
    """Proposal of one k (rows = its active bands).  Without ``log_phi``:
    p(q) = (1 - alpha) mean_rows softmax(logits[row]) + alpha / N_q.  With it (the shell factor):
    p(q) = (1 - alpha) mean_live softmax(logits + log_phi) + alpha mean_live softmax(log_phi) over the
    rows with some phi > 0; the uniform 1/N_q when there is none (every c of the k is then 0)."""
    logits = np.atleast_2d(logits)
    Nq = logits.shape[1]
    if log_phi is None:
        return (1.0 - alpha) * _softmax_rows(logits).mean(axis=0) + alpha / Nq
    lp = np.atleast_2d(log_phi)
    live = np.isfinite(lp).any(axis=1)
    if not live.any():
        return np.full(Nq, 1.0 / Nq)
    return ((1.0 - alpha) * _softmax_rows(logits[live] + lp[live]).mean(axis=0)
            + alpha * _softmax_rows(lp[live]).mean(axis=0))


def shell_proposal(log_phi: np.ndarray) -> np.ndarray:
    """p(q) = mean_live phi_row(q) / sum_q phi_row over the rows with some phi > 0 (uniform if none)."""
    lp = np.atleast_2d(log_phi)
    live = np.isfinite(lp).any(axis=1)
    if not live.any():
        return np.full(lp.shape[1], 1.0 / lp.shape[1])
    return _softmax_rows(lp[live]).mean(axis=0)


def draw(p: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Inverse-CDF draws: the smallest q with CDF(q) > u * CDF(N_q - 1), CDF the FP64 running sum in q order."""
    cdf = np.cumsum(p)
    q = np.searchsorted(cdf, u * cdf[-1], side="right")
    return np.minimum(q, len(p) - 1)


def is_estimate(c_sampled: np.ndarray, p: np.ndarray, q_drawn: np.ndarray) -> np.ndarray:
    """Gamma^ = (1/S) sum_j c(q_j) / (N_q p^(q_j)) with p^ = p / sum p; c_sampled (n_bands, S)."""
    Nq = len(p)
    ph = p / np.sum(p)
    return np.mean(c_sampled / (Nq * ph[q_drawn])[None, :], axis=1)


def linewidths_is(mat, params, blob, fraction: float, alpha: float, seed: int, k_indices=None,
                  uniform: bool = False, table=None, mode: str | None = None):
    """Importance-sampled Gamma of the active states (before degenerate averaging is applied, then
    averaged like ``elph.linewidths_rta``).  ``mode``: "learned" (network times shell factor, the
    default), "shell" (the shell factor alone) or "uniform" (p_k = 1/N_q; also ``uniform=True``).
    Returns (k_index, band, gamma)."""
    mode = "uniform" if uniform else (mode or "learned")
    table = table if table is not None else elph.electron_table(mat, params)
    F, eps_F, U_F, k_to_F = table
    nq = tuple(int(x) for x in params.nq)
    Nq = int(np.prod(nq))
    S = int(np.ceil(fraction * Nq))
    eps_grid = eps_F[k_to_F]
    ks, bs = elph._active(eps_grid, params)
    if k_indices is not None:
        keep = np.isin(ks, np.asarray(k_indices))
        ks, bs = ks[keep], bs[keep]
    theta = bf16_params(blob) if mode == "learned" else None
    qt = wrapped_q(nq)
    feats = state_features(mat, params, ks, bs, table=table) if mode == "learned" else None
    raw = np.zeros(len(ks))
    for ik in np.unique(ks):
        sel = np.nonzero(ks == ik)[0]
        if mode == "uniform":
            p = np.full(Nq, 1.0 / Nq)
        else:
            lp = log_shell(shell_factor(mat, params, ks[sel], bs[sel], table=table))
            if mode == "shell":
                p = shell_proposal(lp)
            else:
                logits = np.stack([mlp_forward(theta, rows_for_state(feats[j], qt))[0] for j in sel])
                p = proposal(logits, alpha, lp)
        q = draw(p, is_uniforms(seed, int(ik), S))
        qi = np.repeat(q[None, :], len(sel), axis=0)
        _, _, c = elph.contributions(mat, params, k_indices=[ik], q_indices=qi, table=table)
        raw[sel] = is_estimate(c, p, q)
    out = raw.copy()
    for ik in np.unique(ks):
        sel = np.nonzero(ks == ik)[0]
        e = eps_grid[ik, bs[sel]]
        for a, j in enumerate(sel):
            grp = sel[np.abs(e - e[a]) < params.degen_tol_eV]
            out[j] = raw[grp].mean()
    return ks, bs, out
