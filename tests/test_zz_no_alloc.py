"""Allocation-free band-energy entry point (phoebe_gpu_bands_noalloc).

It serves callers that cannot allocate device memory: a framework sharing the GPU
may already hold nearly all of it in its own pool, or the device-wide
synchronisation that cudaMalloc/cudaFree may imply is not acceptable.  Checked
here: its energies against the oracle's eigenvalues of H(k) and against the
context path (interpolate_couplings) for the same points; its eigenvectors by the
residual H(k) U = U diag(eps) with H(k) rebuilt by the oracle; two calls in a row
(every call reuses one static scratch array that keeps the previous call's
contents); the U = NULL form; and the size limit at exactly the 16 MiB of scratch
(accepted) and one point beyond it (rejected).
"""
import ctypes
import itertools
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import elph
from workloads import synthetic as W

pytestmark = pytest.mark.gpu

RTOL_FP64 = 1e-10
SCRATCH_BYTES = 16 << 20


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _call(pg, torch, mat, pts, want_U=True):
    """One call through the C ABI on torch's current stream; returns (status, eps, U)."""
    R = _dev(torch, mat.R_H, torch.int32)
    w = _dev(torch, mat.w_H, torch.float64)
    H = _dev(torch, np.ascontiguousarray(mat.H).view(np.float64), torch.float64)
    kd = _dev(torch, pts, torch.float64)
    eps = torch.full((len(pts), mat.nw), np.nan, dtype=torch.float64, device="cuda")
    U = torch.empty((len(pts), mat.nw, mat.nw, 2), dtype=torch.float64, device="cuda") if want_U else None
    stream = torch.cuda.current_stream()
    st = pg.lib.phoebe_gpu_bands_noalloc(mat.nw, len(mat.R_H), ctypes.c_void_p(R.data_ptr()),
                                         ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(H.data_ptr()),
                                         len(pts), ctypes.c_void_p(kd.data_ptr()),
                                         ctypes.c_void_p(eps.data_ptr()),
                                         ctypes.c_void_p(U.data_ptr()) if want_U else None,
                                         ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    Uc = None
    if want_U:
        Uc = U.cpu().numpy()
        Uc = Uc[..., 0] + 1j * Uc[..., 1]
    return st, eps.cpu().numpy(), Uc


def _check_eigenpairs(mat, pts, eps, U):
    """eps against the oracle's eigenvalues; U unitary and H(k) U = U diag(eps)."""
    eps_ref, _ = elph.electron_bands(pts, mat)
    np.testing.assert_allclose(eps, eps_ref, rtol=RTOL_FP64, atol=1e-12)
    Hk = elph.wannier_hamiltonian(pts, mat)
    scale = np.max(np.abs(eps_ref))
    resid = Hk @ U - U * eps[:, None, :]
    assert np.max(np.abs(resid)) < 1e-10 * scale
    eye = np.conj(np.swapaxes(U, 1, 2)) @ U
    assert np.max(np.abs(eye - np.eye(mat.nw))) < 1e-12


def _eight_band_model(seed=5):
    """nw = 8 Hermitian H(R) on {-1,0,1}^3 with H(-R) = H(R)^dagger."""
    rng = np.random.default_rng(seed)
    R = np.array(list(itertools.product((-1, 0, 1), repeat=3)), dtype=np.int32)
    idx = {tuple(r): i for i, r in enumerate(R)}
    minus = np.array([idx[tuple(-r)] for r in R])
    X = (rng.standard_normal((len(R), 8, 8)) + 1j * rng.standard_normal((len(R), 8, 8))) / np.sqrt(2)
    X *= np.exp(-np.linalg.norm(R, axis=1) / 0.7)[:, None, None]
    H = 0.5 * (X + np.conj(np.swapaxes(X[minus], 1, 2)))
    return SimpleNamespace(nw=8, R_H=R, w_H=np.ones(len(R)), H=H)


def test_noalloc_bands_match_oracle_and_context_path_twice():
    import torch
    import paper_2111_14999_b300 as pg

    mat, _ = W.toy(seed=0)
    rng = np.random.default_rng(21)
    k = rng.uniform(-1, 1, (300, 3))
    q = rng.uniform(-1, 1, (300, 3))
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        _, eps_k, eps_kq, _ = ctx.interpolate_couplings(k, q)
    for pts, ref in ((k, eps_k), (k + q, eps_kq)):          # two calls in a row on the shared scratch
        st, eps, U = _call(pg, torch, mat, pts)
        assert st == 0
        np.testing.assert_allclose(eps, ref, rtol=RTOL_FP64, atol=1e-13)
        _check_eigenpairs(mat, pts, eps, U)


def test_noalloc_without_eigenvectors():
    import torch
    import paper_2111_14999_b300 as pg

    mat = _eight_band_model()
    pts = np.random.default_rng(3).uniform(0, 1, (257, 3))
    st, eps_u, U = _call(pg, torch, mat, pts, want_U=True)
    assert st == 0
    _check_eigenpairs(mat, pts, eps_u, U)
    st, eps, _ = _call(pg, torch, mat, pts, want_U=False)
    assert st == 0
    np.testing.assert_array_equal(eps, eps_u)


def test_noalloc_size_limit_is_exact():
    import torch
    import paper_2111_14999_b300 as pg

    mat = _eight_band_model()
    n_max = SCRATCH_BYTES // (2 * 8 * 8 * 16)                # 8192 points at nw = 8 fill the scratch exactly
    assert n_max == 8192
    pts = np.random.default_rng(4).uniform(0, 1, (n_max, 3))
    st, eps, U = _call(pg, torch, mat, pts)
    assert st == 0
    sel = np.random.default_rng(5).choice(n_max, 64, replace=False)
    sel[0], sel[1] = 0, n_max - 1                            # the first and the last point of the scratch
    _check_eigenpairs(mat, pts[sel], eps[sel], U[sel])
    st, eps1, _ = _call(pg, torch, mat, np.vstack([pts, pts[:1]]), want_U=False)
    assert st == -5                                          # PHOEBE_GPU_ERR_NOMEM: one point beyond
    assert np.all(np.isnan(eps1))                            # nothing was launched


def test_noalloc_rejects_bad_arguments_before_launch():
    import paper_2111_14999_b300 as pg
    # 2 * n_k * nw^2 * 16 bytes > 16 MiB: rejected before anything is launched
    st = pg.lib.phoebe_gpu_bands_noalloc(32, 1, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                         1 << 20, ctypes.c_void_p(16), ctypes.c_void_p(16), None, None)
    assert st == -5
    st = pg.lib.phoebe_gpu_bands_noalloc(0, 1, None, None, None, 1, None, None, None, None)
    assert st == -1
