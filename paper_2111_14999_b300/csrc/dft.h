// Stage 2 on grid q points as a separable DFT over the R_p box (dft.cu).
#pragma once

#include "kernels.cuh"

namespace phx {

#ifndef PHX_DFT_LINES
#define PHX_DFT_LINES 8
#endif
#ifndef PHX_DFT_UNIT
#define PHX_DFT_UNIT (PHX_DFT_LINES % 4 == 0 ? 4 : PHX_DFT_LINES % 3 == 0 ? 3 : PHX_DFT_LINES <= 8 ? PHX_DFT_LINES : 1)
#endif
#ifndef PHX_DFT_SPLIT8
#define PHX_DFT_SPLIT8 4
#endif
#ifndef PHX_DFT_THREADS
#define PHX_DFT_THREADS 256
#endif
#ifndef PHX_DFT_MINB
#define PHX_DFT_MINB 2  // blocks per SM the register budget of the one-q kernel is sized for (two Y buffers
                        // keep shared memory at two blocks per SM)
#endif
#ifndef PHX_DFT_MINB2
#define PHX_DFT_MINB2 2  // blocks per SM the register budget of the two-q kernel is sized for
#endif
constexpr int kDftLines = PHX_DFT_LINES;      // jy lines (at one jz) per run of the fused kernel
constexpr int kDftXThreads = PHX_DFT_THREADS;  // threads per block of the fused kernel
constexpr int kDftSplit8 = PHX_DFT_SPLIT8;     // lanes per q of the x sum at nw = 8
constexpr int kDftUnitLines = PHX_DFT_UNIT;   // lines per work unit of the y sum
static_assert(kDftLines % kDftUnitLines == 0 && kDftLines <= 256, "lines per block: a multiple of the y-sum unit, at most 256");

// The R_p set grouped by residues r = R mod N: entries sorted by (rx, ry, rz) residue index,
// "pairs" = distinct (rx, ry), "planes" = distinct rx.
struct DftZArgs {
  // stage-1 GEMM output: row st_kb[s] holds sum_Re w e^{ik.Re} g(Re, Rp)[m][n][sa] (re, im) at
  // column 2 * (((Rp * nw + m) * nw + n) * nm + sa), scaled by 1 / unscale
  const float* X;
  int64_t ldx;
  float unscale;
  const int* st_kb;          // [S] row of X of each state
  const int* st_k;           // [S] k (coarse grid) of each state
  const int* st_b;           // [S] band of each state
  GridMap gm;
  const cplx* UF;            // [NF][nw][nw] eigenvectors U_k[n][b]
  int nw;
  const float* w;            // [nR] R_p weights
  int nR, E, P, Nz, Bz;
  const int* plane_pair_off;  // [Bx+1] first pair of each plane
  const int* pair_ent_off;    // [P+1] first entry of each pair
  const int* ent_az;          // per entry: rz residue index
  const int* ent_r;           // per entry: R_p index
  const float2* Ez;           // [Nz][Bz] e^{2 pi i jz rz / Nz}
  float2* Zs;                 // [S][Nz][P][E] sum_rz Ez[jz][rz] w_R T[R] over the entries of each pair
};

struct DftXArgs {
  const float2* Zs;           // [S][Nz][P][E]
  int P, Bx, By, Nx, Ny, Nz;
  // y groups: the ry residues of x row k (of plane xS[k], and of plane xD[k] for a pair row) grouped
  // as {r, -r mod Ny}.  Group g holds the pair indices (xS[k], r), (xS[k], -r), (xD[k], r), (xD[k], -r),
  // P where a combination is absent (a zero row), and grp_ay[g] = the residue index of r.
  int G;
  const int* row_grp_off;     // [K+1] first group of each x row
  const int4* grp_idx;        // [G]
  const int* grp_ay;          // [G]
  // x rows: the rx residues grouped by r -> -r (mod Nx).  Row k reads Y row xS[k]; a residue
  // with a partner r' = -r (xD[k] >= 0, != xS[k]) has its rows replaced by S = Y_r + Y_r' and
  // D = Y_r - Y_r' and contributes cos(t r) S + i sin(t r) D, t = 2 pi jx / Nx; a residue equal
  // to its negative (r = 0, Nx/2; xD[k] = -1) contributes cos(t r) Y_r; one without a partner
  // (xD[k] == xS[k]) contributes e^{i t r} Y_r in the same form with S = D = Y_r.
  int K, K0, KP;              // rows [0, K0) real-factor, [K0, K0+KP) pairs, the rest without a partner
  const int* xS;              // [K]
  const int* xD;              // [K]
  const float2* Ex;           // [Nx][K] (cos, sin)(2 pi jx r_k / Nx)
  const float2* Ey;           // [Ny][By]
  const int* st_k;            // [S]
  const int* st_b;            // [S]
  const double* epsF;         // [NF][nw]
  GridMap gm;
  const float* epsf;          // [NF][nw] FP32 energies (window test); bands excluded as final states
                              // (final-state window) hold 3e38, out of every reach
  const float4* el4;          // [NF][nw] (eps hi, eps lo, f, 0)
  const float2* UH;           // [NF][nw][nw] conj(U[m][m'])
  const float2* ZT;           // [Nq][nm (v)][nm (sa)] mode factors, transposed
  const float2* omnb;         // [Nq][nm] (omega, n_B)
  float reach, inv_sigma, cut2;
  double scale;               // (2 pi / N_q) / (sqrt(pi) sigma)
  double* gamma;
  int64_t s_base;
  unsigned long long* nq_evaluated;  // [2i] += the (state, q) pairs whose x sum was evaluated
                                     // (i = block % 4); [2i+1] stays 0
  int* err;                   // set to 1 if a bounded wait between the warps of a block ran out
  // phonon-electron rates (optional, nullptr = off): pacc[q][nu] += f(1-f)/kT of the state times
  // sum_m' |g_{m' n nu}(k,q)|^2 e^{-((eps_nk - eps_m'k+q - w_q nu)/sigma)^2}
  double* pacc;
  double mu, inv_kT;
  // adaptive smearing (optional, vel == nullptr = fixed width): hbar v [NF][nw] (vx, vy, vz, 0) in
  // eV A; width = max(sigma_min, sqrt(sum_b (sum_a dv_a cB[a][b])^2 / 12)), cB[a][b] = (b_b)_a / N_b;
  // a state can reach the window when |eps_nk - eps_m'k+q| < omega_max + cut * width
  const float4* vel;
  float cB[9];
  float sigma_min, omega_max, cut;
  // polar long-range term (optional, gL == nullptr = off): g += gL[q][nu] [U_{k+q}^dagger U_k]_{m'n}
  const float2* gL;           // [Nq][nm]
  const cplx* UF;             // [NF][nw][nw] eigenvectors (the initial state's column is staged)
};

// q-only factor of the polar long-range coupling on the q grid (see phoebe_gpu_set_polar).
struct PolarArgs {
  const double* zstar;        // [na][3][3]
  const cplx* Zq;             // [Q][nm][nm] mode factors of Eq. 7
  float2* out;                // [Q][nm]
  int64_t Q;
  int na, nm, N[3], nmax[3];
  double B[9];                // reciprocal rows b_i (1/A), B[3 i + c]
  double eps[9];
  double alpha, cut, pref;    // pref = (4 pi / V) e^2 / (4 pi eps0)
};

// Stage 1 on grid k points as a separable DFT over the R_e box (dft_s1.cu): for the batch's k in
// kx planes, X[row(k)][c] = sum_Re w_e e^{2 pi i k.R_e} g(R_e)[c] with the phase factorised per axis.
// Entries = R_e sorted by (rz, ry) residue pair; pairs sorted by rz residue; z groups {rz, -rz}.
#ifndef PHX_S1_COLS
#define PHX_S1_COLS 64
#endif
constexpr int kS1Cols = PHX_S1_COLS;  // element columns per block
struct S1Args {
  const float2* g;            // [nRe][C] g(R_e)[c] in FP32
  int64_t C;                  // element columns (nRp nw nw 3na)
  float* X;                   // out: row r at X + r ldx, complex values interleaved
  int64_t ldx;                // floats
  int nRe, Pe, Bx, By, Bz, Gz, nkx, nky, nkz;
  const int* ent_row;         // [nRe] R_e index of each entry
  const int* ent_ax;          // [nRe] rx residue index of each entry
  const float* ent_w;         // [nRe] w of each entry
  const int* pair_ent_off;    // [Pe+1]
  const int* pair_ay;         // [Pe] ry residue index of each pair
  const int* rz_pair_off;     // [Bz+1] pairs of each rz residue index
  // y groups of each rz (FP32 form): the pairs of ry residues {r, -r mod Ny} (pair, partner pair),
  // whose rows the kernel replaces by P = W1(r) + W1(-r) and M = W1(r) - W1(-r); a residue equal to
  // its negative or without a partner is a group (pair, pair) of its own
  int Gy;
  const int2* ygrp;           // [Gy]
  const int* ygrp_ay;         // [Gy] ry residue index of the group's first pair
  const int* rz_grp_off;      // [Bz+1] groups of each rz residue index
  const int2* zgrp;           // [Gz] (rz index of r, rz index of -r or -1)
  const float2* Ex;           // [nkx][Bx] e^{2 pi i kx rx / nkx}
  const float2* Ey;           // [nky][By]
  const float2* Ezg;          // [nkz][Gz] e^{2 pi i kz r / nkz} of each group's r
  const int* plane_kx;        // [planes] kx of each plane of the batch
  const int* plane_line_off;  // [planes+1] lines (ky) of each plane
  const int* line_ky;         // [lines]
  const int* line_k_off;      // [lines+1] the batch's k on each line
  const int4* kent;           // [entries] (kz, X row, X row of (kx, ky, -kz) or -1, 0); a k whose -kz
                              // partner is in the batch appears only in its partner's entry
};
size_t s1_smem_bytes(int nRe, int Pe, int Bz, int Gz, int nky, int By, int nkz, int Gy);
// Launches the stage-1 DFT for `planes` kx planes; -1 on a launch error, -2 if Gz > 16 or an X row
// (ldx floats) or g's C columns reach 2^31 elements.
int s1_launch(cudaStream_t st, const S1Args& a, int planes);
// g(R_e)[c] (complex128, [nRe][C]) -> FP32 [nRe][C]
int s1_convert_g(cudaStream_t st, const cplx* g, int64_t n, float2* out);

// ---------------------------------------------------------------- FP64 grid DFT (dft64.cu)
// The same separable evaluation of Eqs. 70-71 as the FP32 kernels, in FP64 throughout: the phase
// tables from sincospi in FP64, g read in complex128, every sum and the Gaussians of Eq. 61 in FP64.
// The index tables (entries, pairs, groups, x rows, batch lines) are the FP32 path's.
constexpr int kS64Cols = 32;    // element columns per block of the FP64 stage 1
constexpr int kDft64Lines = 4;  // jy lines per run of the FP64 y/x kernel
struct S64Args {
  S1Args i;                   // index tables and sizes (its float pointers are unused)
  const double2* g;           // [nRe][C] complex128
  double2* X;                 // out: row r at X + r C
  const double* ent_w;        // [nRe] w of each entry
  const double2* Ex;          // [nkx][Bx]
  const double2* Ey;          // [nky][By]
  const double2* Ezg;         // [nkz][Gz]
};
struct DftZ64Args {
  const double2* X;           // stage-1 rows, row st_kb[s], column ((Rp nw + m) nw + n) 3na + sa
  int64_t ldx;                // complex values per row
  const int* st_kb;
  const int* st_k;
  const int* st_b;
  GridMap gm;
  const cplx* UF;
  int nw;
  const double* w;            // [nR] R_p weights
  int nR, E, P, Nz, Bz;
  const int* plane_pair_off;
  const int* pair_ent_off;
  const int* ent_az;
  const int* ent_r;
  const double2* Ez;          // [Nz][Bz]
  double2* Zs;                // [S][Nz][P][E]
};
struct DftX64Args {
  const double2* Zs;          // [S][Nz][P][E]
  int P, Bx, By, Nx, Ny, Nz;
  int G;
  const int* row_grp_off;
  const int4* grp_idx;
  const int* grp_ay;
  int K, K0, KP;
  const int* xS;
  const int* xD;
  const double2* Ex;          // [Nx][K]
  const double2* Ey;          // [Ny][By]
  const int* st_k;
  const int* st_b;
  GridMap gm;
  int nw, nm;
  const double* epsF;         // [NF][nw]
  const double* fF;           // [NF][nw]
  const cplx* UF;             // [NF][nw][nw]
  const cplx* Zq;             // [Nq][nm (sa)][nm (nu)] mode factors of Eq. 7 (0 for dead modes)
  const double* omega;        // [Nq][nm]
  const double* nB;           // [Nq][nm]
  double reach;               // a final band m' can contribute only if |eps_nk - eps_m'k+q| < reach
  double inv_sigma, xcut;     // 1 / sigma; the Gaussian is 0 for |x| >= xcut = cut sigma
  double scale;               // (2 pi / N_q) / (sqrt(pi) sigma)
  double* gamma;
  int64_t s_base;
  unsigned long long* nq_evaluated;  // [2i] += the evaluated (state, q) pairs, [2i+1] += the
                                     // listed (state, q, band) triples (i = block % 4)
};
size_t s64_smem_bytes(int nRe, int Pe, int Bz, int Gz, int nky, int By, int nkz);
size_t dft64_z_smem_bytes(int ne_plane_max, int E, int Nz, int Bz);
size_t dft64_smem_bytes(int P, int Bx, int By, int E, int Nx, int Ny, int K, int G);
int s64_launch(cudaStream_t st, const S64Args& a, int planes);  // -1 launch error, -2 Gz > 16
int dft64_launch(cudaStream_t st, const DftZ64Args& z, const DftX64Args& x, int S, int ne_plane_max);
int dft_table64(cudaStream_t st, const int* res, int B, int N, double2* E);

// Launches both kernels for S states; -1 on a launch error, -2 for a (nw, 3na) without a kernel.
int dft_launch(cudaStream_t st, const DftZArgs& z, const DftXArgs& x, int S, int nw, int nm, int ne_plane_max);
#ifndef PHX_DFT_QPAIR
#define PHX_DFT_QPAIR 1
#endif
constexpr bool kDftQPair = PHX_DFT_QPAIR != 0;  // two listed q per lane group (lines of Nx >= 32)

// Entries of one run's q list: every q of the run plus, with pairing, one padding entry per
// (warp round, line) at most -- two lines per round of 32 consecutive q when Nx >= 32.
__host__ __device__ constexpr int dft_list_cap(int L, int Nx) { return L * Nx + 2 * ((L * Nx + 31) / 32) + 2; }
// Lanes per q of the x sum for nw Wannier functions.
__host__ __device__ constexpr int dft_split(int nw) { return nw == 8 ? kDftSplit8 : (nw % 2 == 0 ? 2 : 1); }
size_t dft_smem_bytes(int P, int Bx, int By, int nw, int nm, int Nx, int Ny, int K, int G);
size_t dft_z_smem_bytes(int ne_plane_max, int E, int Nz, int Bz);
int dft_table(cudaStream_t st, const int* res, int B, int N, float2* E);
int polar_table(cudaStream_t st, const PolarArgs& a);
// P[q][nu] from pacc (see DftXArgs::pacc); pref = 2 pi / (N_k sqrt(pi) sigma).  -2 if nm > 32.
int prate_finish(cudaStream_t st, const double* acc, const double* omega, const double* nB, int64_t Q, int nm,
                 double pref, double omega_cut, double degen_tol, double* P);
// FP32 tables of the fused kernel from the FP64 band and phonon arrays.
int dft_tables(cudaStream_t st, const double* epsF, const double* fF, int64_t NF, int nw, const cplx* Z,
               const double* om, const double* nB, int64_t Nq, int nm, float* epsf, float4* el4, float2* ZT,
               float2* omnb);

}  // namespace phx
