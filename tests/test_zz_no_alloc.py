"""Allocation-free band-energy entry point against the context-based one.

phoebe_gpu_bands_noalloc serves callers that cannot allocate device memory
(a framework already holds nearly all of it, or cudaMalloc's possible
device-wide synchronisation is not acceptable).  Its eigenvalues must agree
with the band energies the context path (interpolate_couplings) returns for the
same points, on two calls in a row, since every call reuses one static scratch
array that keeps the previous call's contents.
"""
import ctypes

import numpy as np
import pytest

from workloads import synthetic as W

pytestmark = pytest.mark.gpu

RTOL_FP64 = 1e-10


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def test_noalloc_bands_match_context_path_twice():
    import torch
    import paper_2111_14999_b300 as pg

    mat, _ = W.toy(seed=0)
    rng = np.random.default_rng(21)
    k = rng.uniform(-1, 1, (300, 3))
    q = rng.uniform(-1, 1, (300, 3))
    with pg.PhoebeGPU(0) as ctx:
        ctx.set_material(mat)
        _, eps_k, eps_kq, _ = ctx.interpolate_couplings(k, q)

    R = _dev(torch, mat.R_H, torch.int32)
    w = _dev(torch, mat.w_H, torch.float64)
    H = _dev(torch, np.ascontiguousarray(mat.H).view(np.float64), torch.float64)
    stream = torch.cuda.current_stream()
    for pts, ref in ((k, eps_k), (k + q, eps_kq)):          # two calls in a row on the shared scratch
        kd = _dev(torch, pts, torch.float64)
        eps = torch.full((len(pts), mat.nw), np.nan, dtype=torch.float64, device="cuda")
        U = torch.empty((len(pts), mat.nw, mat.nw, 2), dtype=torch.float64, device="cuda")
        st = pg.lib.phoebe_gpu_bands_noalloc(mat.nw, len(mat.R_H), ctypes.c_void_p(R.data_ptr()),
                                             ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(H.data_ptr()),
                                             len(pts), ctypes.c_void_p(kd.data_ptr()),
                                             ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(U.data_ptr()),
                                             ctypes.c_void_p(stream.cuda_stream))
        assert st == 0
        np.testing.assert_allclose(eps.cpu().numpy(), ref, rtol=RTOL_FP64, atol=1e-13)
        Uc = U.cpu().numpy()
        Uc = Uc[..., 0] + 1j * Uc[..., 1]
        eye = np.conj(np.swapaxes(Uc, 1, 2)) @ Uc
        assert np.max(np.abs(eye - np.eye(mat.nw))) < 1e-12


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import paper_2111_14999_b300 as pg
    # 2 * n_k * nw^2 * 16 bytes > 16 MiB: rejected before anything is launched
    st = pg.lib.phoebe_gpu_bands_noalloc(32, 1, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                         1 << 20, ctypes.c_void_p(16), ctypes.c_void_p(16), None, None)
    assert st == -5
    st = pg.lib.phoebe_gpu_bands_noalloc(0, 1, None, None, None, 1, None, None, None, None)
    assert st == -1
