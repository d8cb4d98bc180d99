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

// A (n x n, overwritten) -> eigenvalues ascending in the real parts of A's diagonal, eigenvectors
// as the columns of V (V(:, i) belongs to A(i, i).re).  n <= kMaxNw.  Every intermediate lives in
// A and V, so the two matrices are the solver's only storage: the reflector of step k in column k
// below the diagonal, its beta in A(k, k).im, the complex sub-diagonal t_k in A(k, k+1), the real
// tridiagonal's off-diagonal e_k in A(k+1, k).re.  Returns 0, or 1 if the QR iteration did not
// converge within 30 n steps (A and V then hold no eigenpairs).
__host__ __device__ inline int eigh_hermitian(Strided<cplx> A, Strided<cplx> V, int n) {
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
  // 1. tridiagonalisation; p and q of step k live in row k until the step ends
  for (int k = 0; k + 2 < n; ++k) {
    const cplx x0 = A(k + 1, k);
    double sig = 0.0;
    for (int i = k + 2; i < n; ++i) sig += cabs2(A(i, k));
    if (sig == 0.0) {  // already tridiagonal in this column
      A(k, k + 1) = x0;
      continue;        // beta = A(k, k).im = 0
    }
    const double a0 = sqrt(cabs2(x0)), nx = sqrt(a0 * a0 + sig);
    const cplx ph = a0 > 0.0 ? cplx{x0.re / a0, x0.im / a0} : cplx{1.0, 0.0};
    A(k + 1, k) = {ph.re * (a0 + nx), ph.im * (a0 + nx)};
    const double b = 1.0 / (nx * (nx + a0));
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
    A(k, k + 1) = {-ph.re * nx, -ph.im * nx};  // t_k = alpha
    A(k, k).im = b;
  }
  if (n >= 2) A(n - 2, n - 1) = A(n - 1, n - 2);
  // Q = H_0 ... H_{n-3} by backward accumulation into V
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V(i, j) = {i == j ? 1.0 : 0.0, 0.0};
  for (int k = n - 3; k >= 0; --k) {
    const double b = A(k, k).im;
    if (b == 0.0) continue;
    for (int j = k + 1; j < n; ++j) {
      cplx s = {0.0, 0.0};
      for (int i = k + 1; i < n; ++i) cfma_conja(s, A(i, k), V(i, j));  // v^H V(:, j)
      s = {-b * s.re, -b * s.im};
      for (int i = k + 1; i < n; ++i) {
        cplx x = V(i, j);
        cfma(x, A(i, k), s);
        V(i, j) = x;
      }
    }
  }
  // 2. real tridiagonal: V <- Q D, e_k = |t_k|
  cplx ph = {1.0, 0.0};
  for (int k = 0; k + 1 < n; ++k) {
    const cplx t = A(k, k + 1);
    const double r = sqrt(cabs2(t));
    A(k + 1, k) = {r, 0.0};
    if (r > 0.0) ph = cmul(ph, cplx{t.re / r, t.im / r});
    for (int i = 0; i < n; ++i) V(i, k + 1) = cmul(V(i, k + 1), ph);
  }
  // 3. implicit QR with the Wilkinson shift on w_k = A(k, k).re, e_k = A(k+1, k).re
#define EIGH_W(k) A(k, k).re
#define EIGH_E(k) A((k) + 1, k).re
  constexpr double kEps = 2.220446049250313e-16;
  int hi = n - 1, steps = 0;
  while (hi > 0) {
    int lo = hi;
    while (lo > 0) {
      const double t = fabs(EIGH_E(lo - 1));
      if (t <= kEps * (fabs(EIGH_W(lo - 1)) + fabs(EIGH_W(lo))) || t < 1e-300) {
        EIGH_E(lo - 1) = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {  // w_hi has converged
      --hi;
      continue;
    }
    if (++steps > 30 * n) return 1;
    // shift: the eigenvalue of the trailing 2 x 2 block nearer its last diagonal entry
    const double g = 0.5 * (EIGH_W(hi - 1) - EIGH_W(hi)), f = EIGH_E(hi - 1);
    const double r = sqrt(g * g + f * f);
    const double mu = EIGH_W(hi) - f * f / (g + (g >= 0.0 ? r : -r));
    double x = EIGH_W(lo) - mu, z = EIGH_E(lo);
    double a = EIGH_W(lo), bb = EIGH_E(lo);
    for (int k = lo; k < hi; ++k) {
      // rotation [c s; -s c] on rows/columns (k, k+1) that zeroes z against x
      const double rr = sqrt(x * x + z * z);
      const double c = rr > 0.0 ? x / rr : 1.0, s = rr > 0.0 ? z / rr : 0.0;
      if (k > lo) EIGH_E(k - 1) = rr;
      const double dd = EIGH_W(k + 1);
      const double cc = c * c, ss = s * s, cs = c * s;
      EIGH_W(k) = cc * a + 2.0 * cs * bb + ss * dd;
      const double ek = cs * (dd - a) + (cc - ss) * bb;
      a = ss * a - 2.0 * cs * bb + cc * dd;  // the new w_{k+1}: the next rotation's a
      EIGH_E(k) = ek;
      if (k + 1 < hi) {  // the bulge moves to (k+2, k)
        const double f1 = EIGH_E(k + 1);
        z = s * f1;
        bb = c * f1;  // the new e_{k+1}: the next rotation's b
        x = ek;
      } else {
        EIGH_W(k + 1) = a;
      }
      for (int i = 0; i < n; ++i) {
        const cplx p = V(i, k), q = V(i, k + 1);
        V(i, k) = {c * p.re + s * q.re, c * p.im + s * q.im};
        V(i, k + 1) = {c * q.re - s * p.re, c * q.im - s * p.im};
      }
    }
  }
  // ascending order: selection sort of the diagonal with the columns of V
  for (int i = 0; i + 1 < n; ++i) {
    int best = i;
    for (int j = i + 1; j < n; ++j)
      if (EIGH_W(j) < EIGH_W(best)) best = j;
    if (best != i) {
      const double t = EIGH_W(i);
      EIGH_W(i) = EIGH_W(best);
      EIGH_W(best) = t;
      for (int r = 0; r < n; ++r) {
        const cplx u = V(r, i);
        V(r, i) = V(r, best);
        V(r, best) = u;
      }
    }
  }
#undef EIGH_W
#undef EIGH_E
  return 0;
}

}  // namespace phx
