// Band structures on grids and point lists: Wannier/force-constant Fourier
// sums (Sec. 3.2 Eq. 10, Sec. 3.1 Eq. 3), batched Hermitian eigensolves
// (Eqs. 4, 11; Householder tridiagonalisation and shifted QR), phonon mode factors (Eq. 7), occupations
// (Secs. 4.1-4.2) and the energy window compaction (Sec. 5.2).
//
// Matrices being diagonalised are kept "structure of arrays": element (i,j)
// of matrix b lives at [(i*n + j) * B + b], so a warp touching 32 matrices
// reads 32 consecutive complex numbers.
#include "eigh.cuh"
#include "kernels.cuh"

namespace phx {

// cis[r] = e^{2 pi i r / L}
__global__ void k_cis_table(cplx* cis, int L) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= L) return;
  double s, c;
  sincospi(2.0 * (double)r / (double)L, &s, &c);
  cis[r] = {c, s};
}

// Grid Fourier sum, complex input: out[e][p] = sum_R w_R e^{2 pi i k_p.R} in[R][e] (SoA output),
// evaluated separably over the residue box of R (FP64): on a grid k = (j0/N0, j1/N1, j2/N2) the
// phase factorises per axis, e^{2 pi i k.R} = prod_d e^{2 pi i j_d r_d/N_d}
// with r_d = R_d mod N_d, so out[e][p] = sum_a E0[j0][a] sum_b E1[j1][b] sum_c E2[j2][c] w_R in[R][e]
// over the R of residues (a, b, c).  Three passes: over c for every (a, b) pair present, over b
// into Y[a][e][j1][j2], over a into out.  Equal to the direct sum over R up to rounding.

// e^{2 pi i j r / N} for the residue list res[0..B): E[j][a] (exact integer argument reduction).
__global__ void k_sep_table(const int* __restrict__ res, int B, int N, cplx* __restrict__ E) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * B) return;
  const int j = t / B, a = t % B;
  const int r = (int)(((int64_t)j * res[a]) % N);
  double sv, cv;
  sincospi(2.0 * (double)r / (double)N, &sv, &cv);
  E[t] = {cv, sv};
}

// Zs[pair][e][j2] = sum over the entries of the pair of E2[j2][c] w_R in[R][e]; thread (pair, e, j2).
__global__ void k_sep_z(const cplx* __restrict__ in, const double* __restrict__ w, int E, int npair,
                        const int* __restrict__ pair_off, const int* __restrict__ ent_c, const int* __restrict__ ent_r,
                        const cplx* __restrict__ E2, int N2, int B2, cplx* __restrict__ Zs) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)npair * E * N2) return;
  const int j2 = (int)(t % N2);
  const int e = (int)((t / N2) % E);
  const int pr = (int)(t / ((int64_t)N2 * E));
  cplx acc = {0.0, 0.0};
  for (int i = pair_off[pr]; i < pair_off[pr + 1]; ++i) {
    const int r = ent_r[i];
    const cplx h = ldc(in + (int64_t)r * E + e);
    const double wr = w[r];
    cfma(acc, ldc(E2 + (int64_t)j2 * B2 + ent_c[i]), {h.re * wr, h.im * wr});
  }
  Zs[t] = acc;
}

// Y[a][e][j1][j2] = sum over the pairs (a, b) of E1[j1][b] Zs[pair][e][j2]; thread (a, e, j1, j2).
__global__ void k_sep_y(const cplx* __restrict__ Zs, int E, int B0, const int* __restrict__ plane_off,
                        const int* __restrict__ pair_b, const cplx* __restrict__ E1, int N1, int B1, int N2,
                        cplx* __restrict__ Y) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)B0 * E * N1 * N2) return;
  const int j2 = (int)(t % N2);
  const int j1 = (int)((t / N2) % N1);
  const int e = (int)((t / ((int64_t)N2 * N1)) % E);
  const int a = (int)(t / ((int64_t)N2 * N1 * E));
  cplx acc = {0.0, 0.0};
  for (int pr = plane_off[a]; pr < plane_off[a + 1]; ++pr)
    cfma(acc, ldc(E1 + (int64_t)j1 * B1 + pair_b[pr]), ldc(Zs + ((int64_t)pr * E + e) * N2 + j2));
  Y[t] = acc;
}

// out[e][p] = sum_a E0[j0][a] Y[a][e][j1][j2], p = (j0 * N1 + j1) * N2 + j2; thread (e, p).
__global__ void k_sep_x(const cplx* __restrict__ Y, int E, int B0, const cplx* __restrict__ E0, int N0, int N1,
                        int N2, cplx* __restrict__ out) {
  const int64_t P = (int64_t)N0 * N1 * N2;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)E * P) return;
  const int64_t p = t % P;
  const int e = (int)(t / P);
  const int j0 = (int)(p / ((int64_t)N1 * N2));
  const int64_t l = p % ((int64_t)N1 * N2);
  cplx acc = {0.0, 0.0};
  for (int a = 0; a < B0; ++a) cfma(acc, ldc(E0 + (int64_t)j0 * B0 + a), ldc(Y + ((int64_t)a * E + e) * N1 * N2 + l));
  out[t] = acc;
}

// Inputs of the band-velocity Fourier sums: out[r][a][e] = i R_cart,a H(R)[e] with
// R_cart = sum_i R_i A_i (lattice rows), so that sum_R w_R e^{ik.R} out[R][a] = dH/dk_a.
__global__ void k_vel_input(const cplx* __restrict__ H, const int* __restrict__ R, Lat9 lat, int nR, int E,
                            cplx* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nR * 3 * E) return;
  const int e = (int)(t % E);
  const int a = (int)((t / E) % 3);
  const int r = (int)(t / (3 * (int64_t)E));
  const double x = R[3 * r] * lat.a[a] + R[3 * r + 1] * lat.a[3 + a] + R[3 * r + 2] * lat.a[6 + a];
  const cplx h = H[(int64_t)r * E + e];
  out[t] = {-x * h.im, x * h.re};
}

// hbar v_pb (eV A, Cartesian) = Re (U^dagger dH/dk_a U)_bb (Hellmann-Feynman, Sec. 3.3) from
// dH [a*nw*nw + e][p] (SoA) and U [p][m][b]; thread (p, b); FP32 output (vx, vy, vz, 0).
__global__ void k_band_velocity(const cplx* __restrict__ dH, const cplx* __restrict__ U, int64_t P, int nw,
                                float4* __restrict__ vel) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= P * nw) return;
  const int64_t p = t / nw;
  const int b = (int)(t % nw);
  const int E = nw * nw;
  double v[3] = {0.0, 0.0, 0.0};
  for (int m = 0; m < nw; ++m) {
    const cplx um = U[(p * nw + m) * nw + b];
    for (int n = 0; n < nw; ++n) {
      const cplx un = U[(p * nw + n) * nw + b];
      // conj(um) * un
      const double cr = um.re * un.re + um.im * un.im, ci = um.re * un.im - um.im * un.re;
      for (int a = 0; a < 3; ++a) {
        const cplx d = dH[((int64_t)a * E + m * nw + n) * P + p];
        v[a] += d.re * cr - d.im * ci;
      }
    }
  }
  vel[t] = make_float4((float)v[0], (float)v[1], (float)v[2], 0.f);
}

// Point-list Fourier sum (off-grid k): phases from sincospi(2 frac(k.R)).
__global__ void k_fourier_points_c(const cplx* __restrict__ in, const int* __restrict__ R,
                                   const double* __restrict__ w, int nR, int E,
                                   const double* __restrict__ kpts, int64_t P, cplx* __restrict__ out) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int e = blockIdx.y;
  if (p >= P) return;
  double k0 = kpts[3 * p], k1 = kpts[3 * p + 1], k2 = kpts[3 * p + 2];
  cplx acc = {0.0, 0.0};
  for (int r = 0; r < nR; ++r) {
    double x = k0 * __ldg(R + 3 * r) + k1 * __ldg(R + 3 * r + 1) + k2 * __ldg(R + 3 * r + 2);
    x -= floor(x);
    double s, c;
    sincospi(2.0 * x, &s, &c);
    double wr = __ldg(w + r);
    cfma(acc, {c * wr, s * wr}, ldc(in + (int64_t)r * E + e));
  }
  out[(int64_t)e * P + p] = acc;
}

// Real force constants -> mass-scaled dynamical matrix entry e = (i, j):
// D[e][p] = sum_R w_R Phi[R][e] e^{2 pi i q_p.R} / sqrt(M_i M_j).
__global__ void k_dynmat_grid(const double* __restrict__ Phi, const int* __restrict__ R,
                              const double* __restrict__ w, int nR, int nm,
                              const double* __restrict__ inv_sqrt_m, GridPhase gp,
                              const cplx* __restrict__ cis, const double* __restrict__ qpts,
                              int64_t P, cplx* __restrict__ out) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int e = blockIdx.y;
  if (p >= P) return;
  int E = nm * nm;
  int j[3];
  if (!qpts) grid_coords(p, gp.n, j);
  cplx acc = {0.0, 0.0};
  for (int r = 0; r < nR; ++r) {
    int Rv[3] = {__ldg(R + 3 * r), __ldg(R + 3 * r + 1), __ldg(R + 3 * r + 2)};
    cplx ph;
    if (qpts) {
      double x = qpts[3 * p] * Rv[0] + qpts[3 * p + 1] * Rv[1] + qpts[3 * p + 2] * Rv[2];
      x -= floor(x);
      sincospi(2.0 * x, &ph.im, &ph.re);
    } else {
      ph = ldc(cis + phase_index(j, Rv, gp.mult, gp.L));
    }
    double v = __ldg(Phi + (int64_t)r * E + e) * __ldg(w + r);
    acc.re = fma(v, ph.re, acc.re);
    acc.im = fma(v, ph.im, acc.im);
  }
  double s = inv_sqrt_m[e / nm] * inv_sqrt_m[e % nm];
  out[(int64_t)e * P + p] = {acc.re * s, acc.im * s};
}

// Solved matrix b (eigenvalues ascending on A's diagonal, eigenvectors as V's columns) ->
// evals[b][n], evecs[b][n][n] (eigenvectors as columns).
__device__ __forceinline__ void eigh_store(const Strided<cplx>& a, const Strided<cplx>& v, int n, int64_t b,
                                           double* __restrict__ evals, cplx* __restrict__ evecs) {
  for (int i = 0; i < n; ++i) {
    evals[b * n + i] = a(i, i).re;
    if (evecs)
      for (int k = 0; k < n; ++k) evecs[(b * n + k) * n + i] = v(k, i);
  }
}

// B Hermitian n x n matrices (SoA, in place; V is scratch) -> eigenvalues ascending in
// evals[b][n], eigenvectors as columns in evecs[b][n][n]: one thread per matrix runs the
// Householder tridiagonalisation and shifted QR of eigh_hermitian on its matrix in global memory.
__global__ void k_eigh_herm(cplx* __restrict__ A, cplx* __restrict__ V, int n, int64_t B,
                            double* __restrict__ evals, cplx* __restrict__ evecs, int* __restrict__ status) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= B) return;
  const Strided<cplx> a{A + b, n, B}, v{V + b, n, B};
  if (eigh_hermitian(a, v, n) && status) atomicOr(status, 1);
  eigh_store(a, v, n, b, evals, evecs);
}

int eigh_launch(cudaStream_t st, cplx* A, cplx* V, int n, int64_t B, double* evals, cplx* evecs, int* status) {
  if (B <= 0) return 0;
  // one thread per matrix: small batches in narrow blocks, so that they spread over every SM
  const int T = B <= 148 * 32 ? 32 : B <= 148 * 64 ? 64 : 128;
  k_eigh_herm<<<(unsigned)((B + T - 1) / T), T, 0, st>>>(A, V, n, B, evals, evecs, status);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Phonon energies, Bose factors and mode factors Z = z sqrt(hbar^2/(2 M_s hbar w)) (Eq. 7);
// dead modes (hbar w < omega_cut) get Z = 0 and n = 0.
__global__ void k_phonon_factors(const double* __restrict__ lam, const cplx* __restrict__ z, int nm,
                                 int64_t Q, const double* __restrict__ mass_of_row, double T,
                                 double omega_cut, double* __restrict__ omega, double* __restrict__ nB,
                                 cplx* __restrict__ Z) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Q * nm) return;
  int64_t q = i / nm;
  int nu = (int)(i % nm);
  double l = lam[i];
  double w = kHbarOmegaEV * sqrt(l > 0.0 ? l : 0.0);
  omega[i] = w;
  bool alive = w >= omega_cut;
  nB[i] = alive ? 1.0 / expm1(w / (kBoltzmannEV * T)) : 0.0;
  for (int r = 0; r < nm; ++r) {
    cplx v = z[(q * nm + r) * nm + nu];
    double f = alive ? sqrt(kHbar2AmuEvA2 / (2.0 * mass_of_row[r] * w)) : 0.0;
    Z[(q * nm + r) * nm + nu] = {v.re * f, v.im * f};
  }
}

// f = 1/(e^{(eps-mu)/kT}+1)  (Sec. 4.2)
__global__ void k_fermi(const double* __restrict__ eps, int64_t N, double mu, double T,
                        double* __restrict__ f) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  f[i] = 1.0 / (exp((eps[i] - mu) / (kBoltzmannEV * T)) + 1.0);
}

// ------------------------------------------------------------------ window (Sec. 5.2)
// count[c] = number of bands of candidate k point c (k-grid index kidx[c], or c itself)
// with |eps - mu| < window (all bands if window <= 0).
// Initial-state windows (Sec. 5.2): the population window f(1-f) > delta when delta > 0, else
// the energy window |eps - mu| < window (window <= 0: every state).
__device__ __forceinline__ bool in_window(double e, double mu, double window, double kT, double delta) {
  if (delta > 0.0) {
    const double f = 1.0 / (exp((e - mu) / kT) + 1.0);
    return f * (1.0 - f) > delta;
  }
  return window <= 0.0 || fabs(e - mu) < window;
}

__global__ void k_window_count(const double* __restrict__ epsF, const int* __restrict__ kidx, int64_t NC, int nw, GridMap gm,
                               double mu, double window, double kT, double delta, int* __restrict__ count) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= NC) return;
  int64_t k = kidx ? kidx[c] : c;
  int64_t f = gm.k_to_fine(k);
  int cnt = 0;
  for (int b = 0; b < nw; ++b) {
    double e = epsF[f * nw + b];
    if (in_window(e, mu, window, kT, delta)) ++cnt;
  }
  count[c] = cnt;
}

// Final-state window (Sec. 5.2 applied to both states of a transition): the FP32 energy of every
// band that fails the initial states' window (FP64 test) is replaced by 3e38, so that no state can
// reach it in the window listing of the grid-DFT stage 2.
__global__ void k_final_window(const double* __restrict__ epsF, int64_t n, double mu, double window, double kT,
                               double delta, float* __restrict__ epsf) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  if (!in_window(epsF[t], mu, window, kT, delta)) epsf[t] = 3.0e38f;
}

// Single-block exclusive scan of count[0..N) into offset[0..N], offset[N] = total.
__global__ void k_scan_single_block(const int* __restrict__ count, int64_t N, int64_t* __restrict__ offset) {
  __shared__ int64_t part[1024];
  int t = threadIdx.x;
  int64_t chunk = (N + blockDim.x - 1) / blockDim.x;
  int64_t lo = t * chunk, hi = lo + chunk < N ? lo + chunk : N;
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += count[i];
  part[t] = s;
  __syncthreads();
  for (int d = 1; d < (int)blockDim.x; d <<= 1) {
    int64_t v = (t >= d) ? part[t - d] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int64_t base = part[t] - s;
  for (int64_t i = lo; i < hi; ++i) {
    offset[i] = base;
    base += count[i];
  }
  if (t == blockDim.x - 1) offset[N] = part[t];
}

// Write the active states (k grid index, band) in k-then-band order.
__global__ void k_window_write(const double* __restrict__ epsF, const int* __restrict__ kidx, int64_t NC,
                               int nw, GridMap gm, double mu, double window, double kT, double delta,
                               const int64_t* __restrict__ offset, int* __restrict__ st_k,
                               int* __restrict__ st_b) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= NC) return;
  int64_t k = kidx ? kidx[c] : c;
  int64_t f = gm.k_to_fine(k);
  int64_t o = offset[c];
  for (int b = 0; b < nw; ++b) {
    double e = epsF[f * nw + b];
    if (in_window(e, mu, window, kT, delta)) {
      st_k[o] = (int)k;
      st_b[o] = b;
      ++o;
    }
  }
}

}  // namespace phx
