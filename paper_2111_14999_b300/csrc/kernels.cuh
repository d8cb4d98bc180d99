// Kernel declarations and small host/device structs of the phoebe_gpu library.
#pragma once

#include "common.cuh"

namespace phx {

// Phase lookup on a grid n: k.R = r/L with r = sum_i j_i n_i mult_i (mod L).
struct GridPhase {
  int n[3];
  int mult[3];
  int L;
};

// k grid, q grid and the fine grid holding every k and k+q.
struct GridMap {
  int nk[3], nq[3], nf[3];
  int sk[3], sq[3];  // nf / nk, nf / nq
  __host__ __device__ int64_t k_to_fine(int64_t k) const {
    int c[3];
    grid_coords(k, nk, c);
    int f[3] = {c[0] * sk[0], c[1] * sk[1], c[2] * sk[2]};
    return grid_flat(f, nf);
  }
  __host__ __device__ int64_t kq_to_fine(int64_t k, int64_t q) const {
    int a[3], b[3];
    grid_coords(k, nk, a);
    grid_coords(q, nq, b);
    int f[3];
    for (int i = 0; i < 3; ++i) f[i] = (a[i] * sk[i] + b[i] * sq[i]) % nf[i];
    return grid_flat(f, nf);
  }
};

// ---------------------------------------------------------------- bands.cu
__global__ void k_cis_table(cplx* cis, int L);
struct Lat9 {
  double a[9];  // lattice rows, Cartesian, A
};
__global__ void k_vel_input(const cplx* H, const int* R, Lat9 lat, int nR, int E, cplx* out);
__global__ void k_final_window(const double* epsF, int64_t n, double mu, double window, double kT, double delta,
                               float* epsf);
__global__ void k_band_velocity(const cplx* dH, const cplx* U, int64_t P, int nw, float4* vel);
__global__ void k_sep_table(const int* res, int B, int N, cplx* E);
__global__ void k_sep_z(const cplx* in, const double* w, int E, int npair, const int* pair_off, const int* ent_c,
                        const int* ent_r, const cplx* E2, int N2, int B2, cplx* Zs);
__global__ void k_sep_y(const cplx* Zs, int E, int B0, const int* plane_off, const int* pair_b, const cplx* E1,
                        int N1, int B1, int N2, cplx* Y);
__global__ void k_sep_x(const cplx* Y, int E, int B0, const cplx* E0, int N0, int N1, int N2, cplx* out);
__global__ void k_fourier_points_c(const cplx* in, const int* R, const double* w, int nR, int E,
                                   const double* kpts, int64_t P, cplx* out);
__global__ void k_dynmat_grid(const double* Phi, const int* R, const double* w, int nR, int nm,
                              const double* inv_sqrt_m, GridPhase gp, const cplx* cis, const double* qpts,
                              int64_t P, cplx* out);
__global__ void k_eigh_herm(cplx* A, cplx* V, int n, int64_t B, double* evals, cplx* evecs, int* status);
// Batched Hermitian eigensolve (A, V: [n*n][B] SoA scratch, A overwritten); 0 or -1 on a launch error.
int eigh_launch(cudaStream_t st, cplx* A, cplx* V, int n, int64_t B, double* evals, cplx* evecs, int* status);
__global__ void k_phonon_factors(const double* lam, const cplx* z, int nm, int64_t Q,
                                 const double* mass_of_row, double T, double omega_cut, double* omega,
                                 double* nB, cplx* Z);
__global__ void k_fermi(const double* eps, int64_t N, double mu, double T, double* f);
__global__ void k_window_count(const double* epsF, const int* kidx, int64_t NC, int nw, GridMap gm,
                               double mu, double window, double kT, double delta, int* count);
__global__ void k_scan_single_block(const int* count, int64_t N, int64_t* offset);
__global__ void k_window_write(const double* epsF, const int* kidx, int64_t NC, int nw, GridMap gm,
                               double mu, double window, double kT, double delta, const int64_t* offset, int* st_k,
                               int* st_b);

// ---------------------------------------------------------------- tc_gemm.cu
// *out = bit pattern of max |x_i| (out zeroed by the caller; non-negative doubles order as their bits)
__global__ void k_absmax_f64(const double* x, int64_t n, unsigned long long* out);

// ---------------------------------------------------------------- couple_fp64.cu
__global__ void k_phase_table_grid(cplx* P, const int* pts, int64_t npts, const int* R, const double* w,
                                   int nR, GridPhase gp, const cplx* cis);
__global__ void k_phase_table_points(cplx* P, const double* pts, int64_t npts, const int* R,
                                     const double* w, int nR);
void launch_zgemm(cudaStream_t s, int64_t M, int64_t N, int K, const cplx* A, int64_t lda, const cplx* B,
                  int64_t ldb, cplx* C, int64_t ldc);
__global__ void k_tpack_fp64(const cplx* X, int64_t ldx, const int* st_kb, const int* st_k, const int* st_b,
                             GridMap gm, const cplx* UF, int S, int nRp, int nw, int nm, cplx* T);
__global__ void k_rotate_final_fp64(const cplx* G, int S, int64_t Qc, int64_t q0, const int* st_k,
                                    GridMap gm, const cplx* UF, const cplx* Zq, int nw, int nm,
                                    double* g2);
__global__ void k_delta_accumulate_fp64(const double* g2, int S, int64_t Qc, int64_t q0, const int* st_k,
                                        const int* st_b, int64_t s_base, GridMap gm, const double* epsF,
                                        const double* fF, const double* omega, const double* nB, int nw,
                                        int nm, double sigma, double cut, double pref, double reach,
                                        double* gamma);
__global__ void k_degenerate_average(const double* raw, const int* st_k, const int* st_b, int64_t NS,
                                     const double* epsF, GridMap gm, int nw, double tol, double* out);
__global__ void k_pairs_stage2(const cplx* X, int npairs, const double* q, const int* Rp, const double* wp,
                               int nRp, int nw, int nm, cplx* G);
__global__ void k_pairs_rotate(const cplx* G, int npairs, const cplx* Uk, const cplx* Ukq, const cplx* Zq,
                               int nw, int nm, double* g2);

}  // namespace phx
