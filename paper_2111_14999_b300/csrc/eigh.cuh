// Eigenvalues and eigenvectors of one small Hermitian matrix, for the batched band and phonon
// eigensolves (H(k) of Sec. 3.1, D(q) of Sec. 3.1 Eq. 5).  Three steps:
//  1. Householder reduction to tridiagonal form, A = Q T Q^H, Q = H_0 H_1 ... H_{n-3}.
//     Step k maps x = A[k+1:, k] to alpha e_1 with the Hermitian reflector H = I - beta v v^H,
//     v = x - alpha e_1, alpha = -e^{i arg x_0} |x|, beta = 2 / (v^H v) = 1 / (|x| (|x| + |x_0|)).
//     The trailing block takes the rank-2 update A <- A - v q^H - q v^H with p = beta A v,
//     q = p - (beta/2)(v^H p) v.
//  2. A diagonal unitary D (D_00 = 1, D_{k+1,k+1} = D_kk t_k / |t_k|, t_k the complex
//     sub-diagonal) makes the tridiagonal real: D^H T D has sub-diagonal |t_k|.
//  3. Implicit symmetric QR steps with the Wilkinson shift on the real tridiagonal, each a
//     chain of plane rotations that chases the bulge down the unreduced block; the rotations
//     accumulate into V, which starts as Q D, so V ends as the eigenvector matrix.
// About 10 n^3 real operations instead of the 200 n^3 of a cyclic Jacobi with 6-8 sweeps.
// Host-callable as well, so the arithmetic can be checked on the CPU.
#pragma once

#include "common.cuh"

namespace phx {

// Element (i, j) of an n x n matrix whose entries are s apart (the batched structure-of-arrays
// layout: s = number of matrices).
template <typename T>
struct Strided {
  T* p;
  int n;
  int64_t s;
  __host__ __device__ __forceinline__ T& operator()(int i, int j) const { return p[((int64_t)i * n + j) * s]; }
};

// A (n x n, overwritten) -> eigenvalues w[0..n) in no particular order, eigenvectors as the
// columns of V (V(:, i) belongs to w[i]).  n <= kMaxNw.  Returns 0, or 1 if the QR iteration
// did not converge within 30 n steps (w and V are then not eigenpairs).
__host__ __device__ inline int eigh_hermitian(Strided<cplx> A, Strided<cplx> V, int n, double* w) {
  double beta[kMaxNw], e[kMaxNw];
  cplx off[kMaxNw];
  // exact Hermitian symmetry on entry
  for (int i = 0; i < n; ++i) {
    A(i, i).im = 0.0;
    for (int j = i + 1; j < n; ++j) {
      const cplx u = A(i, j), l = A(j, i);
      const cplx m = {0.5 * (u.re + l.re), 0.5 * (u.im - l.im)};
      A(i, j) = m;
      A(j, i) = {m.re, -m.im};
    }
  }
  // 1. tridiagonalisation; v_k is kept in column k below the diagonal, p and q in row k
  for (int k = 0; k + 2 < n; ++k) {
    const cplx x0 = A(k + 1, k);
    double sig = 0.0;
    for (int i = k + 2; i < n; ++i) sig += cabs2(A(i, k));
    if (sig == 0.0) {  // already tridiagonal in this column
      beta[k] = 0.0;
      off[k] = x0;
      continue;
    }
    const double a0 = sqrt(cabs2(x0)), nx = sqrt(a0 * a0 + sig);
    const cplx ph = a0 > 0.0 ? cplx{x0.re / a0, x0.im / a0} : cplx{1.0, 0.0};
    off[k] = {-ph.re * nx, -ph.im * nx};
    A(k + 1, k) = {ph.re * (a0 + nx), ph.im * (a0 + nx)};
    const double b = 1.0 / (nx * (nx + a0));
    beta[k] = b;
    for (int i = k + 1; i < n; ++i) {  // p = beta A v
      cplx acc = {0.0, 0.0};
      for (int j = k + 1; j < n; ++j) cfma(acc, A(i, j), A(j, k));
      A(k, i) = {b * acc.re, b * acc.im};
    }
    double K = 0.0;  // (beta/2) v^H p, real
    for (int i = k + 1; i < n; ++i) {
      const cplx v = A(i, k), p = A(k, i);
      K += v.re * p.re + v.im * p.im;
    }
    K *= 0.5 * b;
    for (int i = k + 1; i < n; ++i) {  // q = p - K v
      const cplx v = A(i, k), p = A(k, i);
      A(k, i) = {p.re - K * v.re, p.im - K * v.im};
    }
    for (int i = k + 1; i < n; ++i) {  // A <- A - v q^H - q v^H on the lower triangle, mirrored
      const cplx vi = A(i, k), qi = A(k, i);
      for (int j = k + 1; j < i; ++j) {
        const cplx vj = A(j, k), qj = A(k, j);
        const cplx t = cmulc(vi, qj), u = cmulc(qi, vj);
        cplx a = A(i, j);
        a.re -= t.re + u.re;
        a.im -= t.im + u.im;
        A(i, j) = a;
        A(j, i) = {a.re, -a.im};
      }
      const cplx t = cmulc(vi, qi);
      A(i, i) = {A(i, i).re - 2.0 * t.re, 0.0};
    }
  }
  for (int i = 0; i < n; ++i) w[i] = A(i, i).re;
  if (n >= 2) off[n - 2] = A(n - 1, n - 2);
  // Q = H_0 ... H_{n-3} by backward accumulation into V
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V(i, j) = {i == j ? 1.0 : 0.0, 0.0};
  for (int k = n - 3; k >= 0; --k) {
    if (beta[k] == 0.0) continue;
    for (int j = k + 1; j < n; ++j) {
      cplx s = {0.0, 0.0};
      for (int i = k + 1; i < n; ++i) cfma_conja(s, A(i, k), V(i, j));  // v^H V(:, j)
      s = {-beta[k] * s.re, -beta[k] * s.im};
      for (int i = k + 1; i < n; ++i) {
        cplx x = V(i, j);
        cfma(x, A(i, k), s);
        V(i, j) = x;
      }
    }
  }
  // 2. real tridiagonal: V <- Q D
  cplx ph = {1.0, 0.0};
  for (int k = 0; k + 1 < n; ++k) {
    const double r = sqrt(cabs2(off[k]));
    e[k] = r;
    if (r > 0.0) ph = cmul(ph, cplx{off[k].re / r, off[k].im / r});
    for (int i = 0; i < n; ++i) V(i, k + 1) = cmul(V(i, k + 1), ph);
  }
  // 3. implicit QR with the Wilkinson shift; e[k] couples w[k] and w[k+1]
  constexpr double kEps = 2.220446049250313e-16;
  int hi = n - 1, steps = 0;
  while (hi > 0) {
    int lo = hi;
    while (lo > 0) {
      const double t = fabs(e[lo - 1]);
      if (t <= kEps * (fabs(w[lo - 1]) + fabs(w[lo])) || t < 1e-300) {
        e[lo - 1] = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {  // w[hi] has converged
      --hi;
      continue;
    }
    if (++steps > 30 * n) return 1;
    // shift: the eigenvalue of the trailing 2 x 2 block nearer its last diagonal entry
    const double g = 0.5 * (w[hi - 1] - w[hi]), f = e[hi - 1];
    const double r = sqrt(g * g + f * f);
    const double mu = w[hi] - f * f / (g + (g >= 0.0 ? r : -r));
    double x = w[lo] - mu, z = e[lo];
    for (int k = lo; k < hi; ++k) {
      // rotation [c s; -s c] on rows/columns (k, k+1) that zeroes z against x
      const double rr = sqrt(x * x + z * z);
      const double c = rr > 0.0 ? x / rr : 1.0, s = rr > 0.0 ? z / rr : 0.0;
      if (k > lo) e[k - 1] = rr;
      const double a = w[k], bb = e[k], dd = w[k + 1];
      const double cc = c * c, ss = s * s, cs = c * s;
      w[k] = cc * a + 2.0 * cs * bb + ss * dd;
      w[k + 1] = ss * a - 2.0 * cs * bb + cc * dd;
      e[k] = cs * (dd - a) + (cc - ss) * bb;
      if (k + 1 < hi) {  // the bulge moves to (k+2, k)
        z = s * e[k + 1];
        e[k + 1] *= c;
        x = e[k];
      }
      for (int i = 0; i < n; ++i) {
        const cplx p = V(i, k), q = V(i, k + 1);
        V(i, k) = {c * p.re + s * q.re, c * p.im + s * q.im};
        V(i, k + 1) = {c * q.re - s * p.re, c * q.im - s * p.im};
      }
    }
  }
  return 0;
}

}  // namespace phx
