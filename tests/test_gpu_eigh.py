"""The batched Hermitian eigensolver (Householder tridiagonalisation + shifted QR) on
matrices chosen to stress it: repeated eigenvalues, diagonal and already tridiagonal
input, the zero matrix, rank one, a tiny perturbation of a multiple of the identity,
real symmetric input, every size from 1 to 32.

The solver is reached through phoebe_gpu_bands_noalloc with a single lattice vector
R = 0 of weight 1, so that H(k) = H(R=0) at every k: the matrix under test.  Checked
against the definition of an eigendecomposition, not against another solver's
vectors: eigenvalues ascending and equal to LAPACK's (numpy.linalg.eigvalsh) within
1e-13 of the norm, H U = U diag(eps) within 1e-13 of the norm, U^H U = I within 1e-13.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-13


def _matrix(kind, n, rng):
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = 0.5 * (X + X.conj().T)
    if kind == "degenerate":
        Q, _ = np.linalg.qr(X)
        lam = np.round(rng.standard_normal(n)) * 0.5  # few distinct values, many repeats
        A = (Q * lam) @ Q.conj().T
    elif kind == "diagonal":
        A = np.diag(rng.standard_normal(n)).astype(complex)
    elif kind == "zero":
        A = np.zeros((n, n), complex)
    elif kind == "tridiagonal":
        A = A * (np.abs(np.subtract.outer(np.arange(n), np.arange(n))) <= 1)
    elif kind == "rank_one":
        v = X[:, :1]
        A = v @ v.conj().T
    elif kind == "near_identity":
        A = 3.0 * np.eye(n) + 1e-9 * A
    elif kind == "real":
        A = A.real.astype(complex)
    return 0.5 * (A + A.conj().T)


def _eigh_gpu(pg, torch, A, n_k=3):
    n = A.shape[0]
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)
    R = dev(np.zeros((1, 3), np.int32), torch.int32)
    w = dev(np.ones(1), torch.float64)
    H = dev(np.ascontiguousarray(A[None]).view(np.float64), torch.float64)
    k = dev(np.random.default_rng(0).random((n_k, 3)), torch.float64)
    eps = torch.full((n_k, n), np.nan, dtype=torch.float64, device="cuda")
    U = torch.empty((n_k, n, n, 2), dtype=torch.float64, device="cuda")
    st = pg.lib.phoebe_gpu_bands_noalloc(n, 1, ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                         ctypes.c_void_p(H.data_ptr()), n_k, ctypes.c_void_p(k.data_ptr()),
                                         ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(U.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    Uc = U.cpu().numpy()
    return st, eps.cpu().numpy(), Uc[..., 0] + 1j * Uc[..., 1]


@pytest.mark.parametrize("kind", ["random", "degenerate", "diagonal", "zero", "tridiagonal", "rank_one",
                                  "near_identity", "real"])
def test_eigh_definition(kind):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2111_14999_b300 as pg
    rng = np.random.default_rng(11)
    for n in range(1, 33):
        A = _matrix(kind, n, rng)
        st, eps, U = _eigh_gpu(pg, torch, A)
        assert st == 0, (kind, n, st)
        scale = max(np.linalg.norm(A, 2), 1e-300)
        ref = np.linalg.eigvalsh(A)
        for i in range(len(eps)):
            assert np.all(np.diff(eps[i]) >= 0), (kind, n)
            assert np.max(np.abs(eps[i] - ref)) <= TOL * scale + 1e-300, (kind, n)
            assert np.max(np.abs(U[i].conj().T @ U[i] - np.eye(n))) <= TOL, (kind, n)
            assert np.max(np.abs(A @ U[i] - U[i] * eps[i])) <= TOL * scale + 1e-300, (kind, n)
        # every k carries the same matrix: the same result from every thread
        assert np.array_equal(eps[0], eps[-1]) and np.array_equal(U[0], U[-1])
