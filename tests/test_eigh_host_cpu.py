"""The batched eigensolver's arithmetic on the CPU (no GPU needed): `csrc/eigh.cuh` is host-callable,
so a small wrapper compiled with nvcc for the host runs the exact code the GPU kernel runs, on the
same structure-of-arrays layout.  Checked against the definition of an eigendecomposition, with
LAPACK's eigenvalues (numpy.linalg.eigvalsh) as the reference spectrum: every size 1-32, random,
degenerate, diagonal, zero, tridiagonal, rank-one, near-identity and real matrices; eigenvalues
ascending and within 1e-13 of the norm, H U = U diag(eps) and U^H U = I within 1e-13."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2111_14999_b300", "csrc")
TOL = 1e-13

WRAPPER = r"""
#include "eigh.cuh"
using namespace phx;
extern "C" int host_eigh(int n, int B, double* a_soa, double* w, double* v_soa) {
  cplx* A = reinterpret_cast<cplx*>(a_soa);
  cplx* V = reinterpret_cast<cplx*>(v_soa);
  int bad = 0;
  for (int b = 0; b < B; ++b) {
    Strided<cplx> a{A + b, n, B}, v{V + b, n, B};
    bad += eigh_hermitian(a, v, n);
    for (int i = 0; i < n; ++i) w[(size_t)b * n + i] = a(i, i).re;
  }
  return bad;
}
"""


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("eigh_host")
    src, so = d / "host_eigh.cu", d / "libhost_eigh.so"
    src.write_text(WRAPPER)
    subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-I", CSRC, "-o", str(so),
                    str(src)], check=True, capture_output=True)
    return ctypes.CDLL(str(so))


def _solve(lib, mats):
    B, n, _ = mats.shape
    soa = np.ascontiguousarray(np.transpose(mats, (1, 2, 0))).astype(np.complex128)  # [i][j][b]
    a = soa.view(np.float64).copy()
    v = np.zeros_like(a)
    w = np.zeros((B, n))
    P = ctypes.POINTER(ctypes.c_double)
    bad = lib.host_eigh(n, B, a.ctypes.data_as(P), w.ctypes.data_as(P), v.ctypes.data_as(P))
    V = v.view(np.complex128).reshape(n, n, B).transpose(2, 0, 1)
    return bad, w, V


def _matrices(kind, n, rng, B=8):
    X = rng.standard_normal((B, n, n)) + 1j * rng.standard_normal((B, n, n))
    A = 0.5 * (X + X.conj().transpose(0, 2, 1))
    if kind == "degenerate":
        Q, _ = np.linalg.qr(X)
        lam = np.round(rng.standard_normal((B, n))) * 0.5
        A = Q @ (lam[:, :, None] * Q.conj().transpose(0, 2, 1))
    elif kind == "diagonal":
        A = np.zeros_like(A)
        A[:, range(n), range(n)] = rng.standard_normal((B, n))
    elif kind == "zero":
        A = np.zeros_like(A)
    elif kind == "tridiagonal":
        A = A * (np.abs(np.subtract.outer(np.arange(n), np.arange(n))) <= 1)
    elif kind == "rank_one":
        u = X[:, :, :1]
        A = u @ u.conj().transpose(0, 2, 1)
    elif kind == "near_identity":
        A = 3.0 * np.eye(n) + 1e-9 * A
    elif kind == "real":
        A = A.real.astype(np.complex128)
    return 0.5 * (A + A.conj().transpose(0, 2, 1))


@pytest.mark.parametrize("kind", ["random", "degenerate", "diagonal", "zero", "tridiagonal", "rank_one",
                                  "near_identity", "real"])
def test_eigh_host_definition(lib, kind):
    rng = np.random.default_rng(7)
    for n in range(1, 33):
        A = _matrices(kind, n, rng)
        bad, w, V = _solve(lib, A)
        assert bad == 0, (kind, n)
        scale = np.maximum(np.linalg.norm(A, 2, axis=(1, 2)), 1e-300)
        ref = np.linalg.eigvalsh(A)
        assert np.all(np.diff(w, axis=1) >= 0), (kind, n)
        assert np.all(np.max(np.abs(w - ref), axis=1) <= TOL * scale + 1e-300), (kind, n)
        eye = V.conj().transpose(0, 2, 1) @ V
        assert np.max(np.abs(eye - np.eye(n))) <= TOL, (kind, n)
        resid = np.max(np.abs(A @ V - V * w[:, None, :]), axis=(1, 2))
        assert np.all(resid <= TOL * scale + 1e-300), (kind, n)
