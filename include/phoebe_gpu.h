/*
 * phoebe_gpu.h -- C ABI of the B300 (sm_103a) el-ph coupling interpolation and
 * RTA linewidth library.
 *
 * What it computes (arXiv 2111.14999):
 *   - electronic bands by Wannier interpolation, H^W_k = sum_R e^{ik.R} <0n|H|Rm>,
 *     U_k^dagger H^W_k U_k = diag(eps_k)                         (Sec. 3.2, Eqs. 10-11)
 *   - phonons from the dynamical matrix, D(q) z = (hbar w)^2 z     (Sec. 3.1, Eqs. 3-4)
 *   - el-ph couplings interpolated from the Wannier representation
 *     g(k,q) = U_{k+q}^dagger [sum_{Re,Rp} e^{i(k.Re + q.Rp)} g(Re,Rp)] U_k z_q / sqrt(2 M w)
 *                                                                  (Sec. 3.2, Eqs. 7 and 13;
 *                                                                   factorised as Sec. 5.5, Eqs. 70-71)
 *   - RTA linewidths Gamma_nk = hbar/tau_nk, Gaussian-smeared        (Sec. 4.2 Eq. 29, Sec. 4.7 Eq. 61)
 *
 * Units: energies eV, lengths Angstrom, masses amu, force constants eV/A^2,
 * Wannier couplings eV/A, output couplings eV.  k, q are crystal (fractional)
 * coordinates; R are integer lattice coordinates; k.R = 2 pi sum_i k_i n_i.
 *
 * Conventions shared by every entry point:
 *   - Every function returns a phoebe_gpu_status; none aborts or exits.  The
 *     text of the last error of a context is returned by phoebe_gpu_last_error.
 *   - Host buffers are owned by the caller.  set_* copy them into device memory
 *     owned by the context before returning; outputs go to caller buffers.
 *   - A context belongs to one device and one CUDA stream and is not
 *     thread-safe.  All work of a call is ordered on that stream.
 *   - Complex arrays are interleaved (re, im) pairs of double.
 *   - Every wait inside a kernel is bounded; a wait that runs out returns
 *     PHOEBE_GPU_ERR_TIMEOUT and leaves the context usable.
 */
#ifndef PHOEBE_GPU_H
#define PHOEBE_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct phoebe_gpu_ctx phoebe_gpu_ctx;

typedef enum {
  PHOEBE_GPU_OK = 0,
  PHOEBE_GPU_ERR_ARG = -1,            /* NULL pointer, non-positive size, bad enum value */
  PHOEBE_GPU_ERR_ORDER = -2,          /* a required set_* call has not been made */
  PHOEBE_GPU_ERR_SHAPE = -3,          /* sizes of the set_* inputs disagree with each other */
  PHOEBE_GPU_ERR_GRID = -4,           /* k and q grids not commensurate, or a bad k_subset index */
  PHOEBE_GPU_ERR_NOMEM = -5,          /* device allocation failed or exceeds the memory cap */
  PHOEBE_GPU_ERR_CUDA = -6,           /* a CUDA runtime call failed (text in last_error) */
  PHOEBE_GPU_ERR_TIMEOUT = -7,        /* a bounded device-side wait ran out */
  PHOEBE_GPU_ERR_NOTCONVERGED = -8,   /* an eigensolve hit its QR step cap */
  PHOEBE_GPU_ERR_UNSUPPORTED = -9     /* valid request the library does not implement */
} phoebe_gpu_status;

typedef enum {
  PHOEBE_PREC_FP64 = 0,        /* every step in FP64 */
  PHOEBE_PREC_SPLIT_BF16 = 1,  /* R_e and R_p phase contractions on tcgen05 tensor cores with each
                                  FP32 operand split into three BF16 parts (hi + mid + lo) and the six
                                  leading cross products, FP32 accumulate; eigensolves, occupations,
                                  the delta arguments and the Gamma reduction in FP64 */
  PHOEBE_PREC_SPLIT_TF32 = 2,  /* same with two TF32 parts (big + small) and three products */
  PHOEBE_PREC_BF16 = 3,        /* single-pass BF16 contractions (reported, not within 1e-5) */
  PHOEBE_PREC_TF32 = 4,        /* single-pass TF32 contractions (reported, not within 1e-5) */
  PHOEBE_PREC_SPLIT_FP16 = 5,  /* two FP16 parts (hi + lo) of power-of-two scaled operands, three
                                  products: 22 significant bits at the cost of three BF16 passes */
  PHOEBE_PREC_BF16X3 = 6,      /* two BF16 parts, three products (reported, ~1e-5) */
  PHOEBE_PREC_FP32_DFT = 7     /* linewidths only: both phase sums on the grids as separable DFTs
                                  over the R residues mod the grid sizes (e^{ik.R} factorises per
                                  axis on a grid): stage 1 over the k grid (the SPLIT_FP16 GEMM when
                                  the R_e residue tables do not fit), stage 2 for the q whose final
                                  bands can reach the delta window, FP32 on the CUDA cores,
                                  rotations and deltas fused; needs q-grid size Nx <= 256,
                                  nw in {1, 2, 4, 8} and 3na in {3, 6} */,
  PHOEBE_PREC_FP64_DFT = 8     /* linewidths only: the separable grid DFTs of PHOEBE_PREC_FP32_DFT in
                                  FP64 throughout (phase tables, both stages, rotations, Gaussians),
                                  the plain FP64 counterpart of the same algorithm; fixed smearing,
                                  full q sum, no polar term or phonon-electron rates; needs the
                                  stage-1 residue tables in shared memory, nw <= 16, 3na <= 30 */
} phoebe_gpu_precision;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (may be NULL: the context creates its own non-blocking stream).  The
 * library never destroys a stream it did not create. */
int phoebe_gpu_create(phoebe_gpu_ctx** out, int device, void* cuda_stream);
/* Release every device buffer of the context.  NULL is accepted. */
int phoebe_gpu_destroy(phoebe_gpu_ctx* ctx);
/* Text of the last error raised on this context ("" if none).  Valid until the next call. */
const char* phoebe_gpu_last_error(const phoebe_gpu_ctx* ctx);

/* Electronic Hamiltonian in the Wannier basis (Sec. 3.2, Eq. 10).
 *   nw  number of Wannier functions, 1..32
 *   R   n_R x 3 int32 lattice coordinates; the set must be closed under -R
 *   w   n_R weights (Wigner-Seitz 1/degeneracy) or NULL for all 1
 *   H   n_R x nw x nw complex (re,im doubles), H[R][n][m] = <0 n|H|R m> in eV;
 *       H(-R) must equal H(R)^dagger so that H^W_k is Hermitian.
 * Replaces any previous Hamiltonian and invalidates cached band structures. */
int phoebe_gpu_set_hamiltonian(phoebe_gpu_ctx* ctx, int nw, int n_R, const int32_t* R,
                               const double* w, const double* H);

/* Harmonic force constants (Sec. 3.1, Eq. 3).
 *   na        atoms per cell, 1..10 (3*na phonon modes)
 *   mass_amu  na masses in amu
 *   R, w      n_R lattice vectors (int32 x3) and weights (NULL = 1)
 *   Phi       n_R x (3na) x (3na) real, eV/A^2, Phi[R][s*3+a][s'*3+b] = d2E/du(s a 0)du(s' b R).
 * The dynamical matrix is mass-scaled: D = sum_R w_R Phi(R) e^{iq.R} / sqrt(M_s M_s'). */
int phoebe_gpu_set_force_constants(phoebe_gpu_ctx* ctx, int na, const double* mass_amu, int n_R,
                                   const int32_t* R, const double* w, const double* Phi);

/* Primitive lattice vectors (rows, Cartesian, Angstrom; lattice[3*i + a] = a-th component of
 * vector i), needed by the adaptive smearing (band velocities in Cartesian coordinates and the
 * reciprocal vectors).  ERR_ARG for a singular lattice. */
int phoebe_gpu_set_lattice(phoebe_gpu_ctx* ctx, const double* lattice);

/* Polar long-range coupling (Sec. 3.2, Eq. polarlong), added to the interpolated g before |g|^2:
 *   g^L_{m'n nu}(k,q) = L_{q nu} [U_{k+q}^dagger U_k]_{m'n},
 *   L_{q nu} = i (4 pi/V) e^2/(4 pi eps0) sum_s sum_{G, q+G != 0} [(q+G).Z*_s.Z_q[s.][nu]] /
 *              [(q+G).eps_inf.(q+G)] exp(-(q+G).eps_inf.(q+G) / (4 alpha)),
 * Z_q the mode factors of Eq. 7 (A), V the cell volume, terms with exponent >= 25 dropped.
 *   Zstar    na x 3 x 3 Born effective charges (Zstar[s][a][b], row a contracted with q+G)
 *   eps_inf  3 x 3 high-frequency dielectric tensor (symmetric positive definite)
 *   alpha    Gaussian filter, 1/A^2 (> 0); Zstar == NULL switches the term off.
 * Needs set_force_constants (na) and set_lattice; used by linewidths_rta with precision
 * PHOEBE_PREC_FP32_DFT (ERR_UNSUPPORTED for other precisions, sampled q sums, adaptive smearing
 * and phonon_rates_elph while it is on). */
int phoebe_gpu_set_polar(phoebe_gpu_ctx* ctx, const double* Zstar, const double* eps_inf, double alpha);

/* Electron-phonon coupling in the Wannier representation (Sec. 3.2, Eq. 13).
 *   Re, we  n_Re electron lattice vectors and weights (NULL = 1)
 *   Rp, wp  n_Rp phonon lattice vectors and weights (NULL = 1)
 *   g       n_Re x n_Rp x nw(m) x nw(n) x 3na complex, eV/A.  m is the k+q (final-state)
 *           Wannier index, n the k (initial-state) index.  Any 1/N_e normalisation of
 *           Eq. 13 is folded into g.
 * Requires set_hamiltonian (for nw) and set_force_constants (for na) first. */
int phoebe_gpu_set_elph_wannier(phoebe_gpu_ctx* ctx, int n_Re, const int32_t* Re, const double* we,
                                int n_Rp, const int32_t* Rp, const double* wp, const double* g);

/* Couplings at explicit (k, q) pairs (need not lie on a grid).
 *   k, q     n_pairs x 3 crystal coordinates
 *   precision  PHOEBE_PREC_FP64 only (others return ERR_UNSUPPORTED)
 *   g2       n_pairs x nw(m') x nw(n) x 3na |g_{m' n nu}(k,q)|^2 in eV^2 (or NULL)
 *   eps_k, eps_kq  n_pairs x nw band energies at k and k+q, ascending (or NULL)
 *   omega_q  n_pairs x 3na phonon energies hbar w in eV, ascending (or NULL)
 * Eigenvector phases are arbitrary, so only gauge-invariant combinations of g2
 * (sums over degenerate subspaces) are meaningful.  Modes with hbar w below
 * 1e-4 eV get g2 = 0. */
int phoebe_gpu_interpolate_couplings(phoebe_gpu_ctx* ctx, int n_pairs, const double* k, const double* q,
                                     int precision, double* g2, double* eps_k, double* eps_kq,
                                     double* omega_q);

typedef struct {
  int nk[3], nq[3];          /* Gamma-centred grids; per axis one of nk[i], nq[i] divides the other */
  double T_K;                /* temperature, K (> 0) */
  double mu_eV;              /* chemical potential */
  double sigma_eV;           /* Gaussian smearing width (> 0), Eq. 61 */
  double window_eV;          /* initial states with |eps - mu| < window; <= 0: all states */
  double delta_cut_sigmas;   /* delta(x) = 0 for |x| >= cut*sigma (default 6) */
  double omega_cut_eV;       /* modes with hbar w < cut contribute nothing (default 1e-4) */
  double degen_tol_eV;       /* Gamma averaged over bands within tol at the same k (default 1e-6) */
  int precision;             /* phoebe_gpu_precision */
  int n_k_subset;            /* > 0: restrict initial k points to k_subset (host, ascending, unique) */
  const int32_t* k_subset;   /*       k-grid indices (i1*N2+i2)*N3+i3 */
  int max_batch_states;      /* states per stage-1/stage-2 batch, 0 = automatic */
  int sampler;               /* phoebe_gpu_sampler: how the q sum of Eq. 29 is evaluated (default full) */
  double sample_fraction;    /* sampler LEARNED/UNIFORM/SHELL: draws per initial k = ceil(fraction * N_q),
                                0 < fraction <= 1 (default 0.05) */
  double mix_alpha;          /* sampler LEARNED: weight of the shell-only part of the proposal,
                                0 < alpha <= 1 (default 0.1) */
  uint64_t seed;             /* sampler LEARNED/UNIFORM/SHELL: key of the Philox4x32-10 draws */
  int sampler_fp32_network;  /* sampler LEARNED: 1 scores q with the FP32 CUDA-core forward pass,
                                0 (default) with the tensor-core kernel (FP16 operands) on sm_10x */
  int smearing;              /* 0 (default): Gaussian of fixed width sigma_eV; 1: adaptive width per pair
                                of states (Sec. 4.7), sigma = max(sigma_min_eV, (1/sqrt 12) sqrt(sum_b
                                ((hbar v_nk - hbar v_m'k+q) . b_b / N_b)^2)), b_b the reciprocal vectors,
                                N_b the q grid; needs phoebe_gpu_set_lattice and precision
                                PHOEBE_PREC_FP32_DFT */
  double population_delta;   /* > 0: initial states are those with f(1 - f) > population_delta (the
                                population window of Sec. 5.2, 0 < delta < 1/4) instead of the energy
                                window; 0 (default): energy window */
  double sigma_min_eV;       /* adaptive smearing: floor of the width (> 0, default 1e-3) */
  int window_final;          /* 1: final states (k+q, m') must also pass the window (energy or
                                population, as the initial states); 0 (default): every band at k+q.
                                1 needs precision PHOEBE_PREC_FP32_DFT */
  int reserved1;             /* must be zero */
} phoebe_gpu_rta_params;

typedef enum {
  PHOEBE_SAMPLER_FULL = 0,     /* every q of the grid (the paper's sum) */
  PHOEBE_SAMPLER_LEARNED = 1,  /* importance sampling from the learned proposal (see below) */
  PHOEBE_SAMPLER_UNIFORM = 2,  /* importance sampling from the uniform proposal */
  PHOEBE_SAMPLER_SHELL = 3     /* importance sampling from the shell factor alone (no network) */
} phoebe_gpu_sampler;

/* Fill *p with the defaults (cut 6 sigma, omega_cut 1e-4, degen 1e-6, FP64, T=300, full q sum,
 * sample fraction 0.05, alpha 0.1, seed 0, fixed smearing, sigma_min 1e-3). */
void phoebe_gpu_rta_params_default(phoebe_gpu_rta_params* p);

/* RTA linewidths of all active (k, n) states on the k grid (Sec. 4.2 Eq. 29):
 *   Gamma_nk = (2 pi/N_q) sum_{q m' nu} |g_{m' n nu}(k,q)|^2
 *              [(n_{q nu} + 1 - f_{m',k+q}) delta(eps_nk - hbar w_{q nu} - eps_{m',k+q})
 *             + (n_{q nu} + f_{m',k+q})     delta(eps_nk + hbar w_{q nu} - eps_{m',k+q})]
 * in eV, k+q looked up on the finer of the two grids, then averaged over
 * degenerate active bands at the same k.
 * Two-call pattern: with gamma_eV == NULL only *n_states is written.  Otherwise
 * *n_states must hold the capacity of the outputs on entry (ERR_ARG if too
 * small) and holds the count on return.  Outputs (host, caller-owned): k_index
 * (grid index), band (0-based, ascending energy), gamma_eV; ordered by k then
 * band.  k_index/band may be NULL. */
int phoebe_gpu_linewidths_rta(phoebe_gpu_ctx* ctx, const phoebe_gpu_rta_params* params, int* n_states,
                              int32_t* k_index, int32_t* band, double* gamma_eV);
/* Same with device output buffers (on the context's device), written in stream order;
 * the call returns after the work is queued and *n_states is known. */
int phoebe_gpu_linewidths_rta_dev(phoebe_gpu_ctx* ctx, const phoebe_gpu_rta_params* params, int* n_states,
                                  int32_t* k_index_dev, int32_t* band_dev, double* gamma_dev);

/* Phonon-electron scattering rates on the q grid (Sec. 4.3, the phonon-electron term on the
 * diagonal of the phonon scattering matrix), with the paper's replacement
 * f_kb - f_{k+q b'} -> (df/deps)(eps_kb) hbar w_{q nu}:
 *   P_{q nu} = (2 pi / N_k) n_{q nu} (n_{q nu} + 1) hbar w_{q nu}
 *              sum_{k b b'} |g_{b' b nu}(k,q)|^2 [f (1 - f) / k_B T]_{kb} delta(eps_kb - eps_{k+q b'} - hbar w_{q nu})
 * in eV, b over the active initial states of the window (as linewidths_rta), b' over all bands,
 * delta the truncated Gaussian, 0 for dead modes, averaged over modes degenerate within
 * degen_tol at the same q.  Runs the whole linewidth pipeline once (Gamma is computed along the
 * way and discarded); params->precision must be PHOEBE_PREC_FP32_DFT and the sampler FULL
 * (ERR_UNSUPPORTED otherwise).  P_eV: host, caller-owned, n_values = N_q * 3 n_at doubles in
 * q-grid order, [q][nu] (ERR_ARG on another count). */
int phoebe_gpu_phonon_rates_elph(phoebe_gpu_ctx* ctx, const phoebe_gpu_rta_params* params, int64_t n_values,
                                 double* P_eV);

/* Third-order force constants V3(s a R, s' b R', s'' c 0) (Sec. 3.1) on n (R, R') pairs:
 *   R, Rp  n x 3 lattice vectors (crystal coordinates), w  n weights (NULL = 1),
 *   Phi3   n x (3na) x (3na) x (3na) real, eV/A^3, [s a][s' b][s'' c]; any 1/N0^3 folded in.
 * Requires set_force_constants (na) first. */
int phoebe_gpu_set_force_constants3(phoebe_gpu_ctx* ctx, int n, const int32_t* R, const int32_t* Rp, const double* w,
                                    const double* Phi3);

/* Three-phonon part of the diagonal of the phonon scattering matrix on the q grid params->nq
 * (Sec. 4.3, with the coupling V3 of Sec. 3.1 interpolated on the grid):
 *   A_{q nu} = (2 pi / N_q) sum_{q~ nu' nu''} |V3(q nu, q~ nu', -(q+q~) nu'')|^2
 *              [n n' (n''+1) delta(w + w' - w'') + (1/2) n (n'+1)(n''+1) delta(w - w' - w'')]
 * (coalescence with q' = q~ plus half the decay with q' = -q~, q'' = q + q~), in eV, with the
 * mode factors of Eq. 7, the Gaussian of fixed width sigma_eV, dead modes excluded, averaged
 * over degenerate modes.  Uses nq, T_K, sigma_eV, delta_cut_sigmas, omega_cut_eV, degen_tol_eV
 * of params.  One or two atoms, N_q <= 65535.  A_eV: host, n_values = N_q * 3na doubles, [q][nu]. */
int phoebe_gpu_three_phonon_rates(phoebe_gpu_ctx* ctx, const phoebe_gpu_rta_params* params, int64_t n_values,
                                  double* A_eV);

/* Work and timing record of the last linewidths_rta call. */
typedef struct {
  int64_t n_states;            /* active states computed */
  int64_t n_k;                 /* distinct initial k points */
  int64_t n_q;                 /* q points */
  int64_t pairs_dense;         /* sum over states of N_q */
  int64_t pairs_executed;      /* (state, q) pairs whose contraction ran */
  int64_t couplings_dense;     /* pairs_dense * nw * 3na */
  int64_t couplings_executed;  /* pairs_executed * nw * 3na */
  int64_t kernel_launches;     /* kernels this library launched in the call */
  int64_t stage2_launches;     /* launches of the dominant (R_p contraction) kernel */
  double stage2_flops;         /* real flops of the R_p contraction as evaluated, 8 per complex MAC:
                                  8 N_Rp nw 3na per pair for the GEMM forms, the DFT's MACs for
                                  PHOEBE_PREC_FP32_DFT */
  double stage2_ms;            /* event-timed device time of the R_p contraction launches */
  double bands_ms, phonons_ms, window_ms, stage1_ms, rotate_ms, delta_ms, total_ms;
  double sampler_ms;           /* sampled q sums: network scores, proposal and draws */
} phoebe_gpu_stats;

/* Turn per-stage event timing on (1) or off (0, default). */
int phoebe_gpu_set_profiling(phoebe_gpu_ctx* ctx, int on);
int phoebe_gpu_get_stats(const phoebe_gpu_ctx* ctx, phoebe_gpu_stats* out);

/* Cap on the context's device memory (bytes, 0 = none); exceeding it returns ERR_NOMEM. */
int phoebe_gpu_set_memory_cap(phoebe_gpu_ctx* ctx, int64_t bytes);

/* RTA transport coefficients from the linewidths of linewidths_rta with the same parameters
 * (Sec. 4.2 fluxes J and Q, Onsager coefficients; Sec. 4.3.2): with tau = hbar / Gamma and hbar v
 * the k-derivative of Eq. 10 (Sec. 3.3, Cartesian),
 *     L_n = 1/(N_k V) sum_{active kb, Gamma > 0} tau v v^T (eps - mu)^n (-df/deps),
 *     sigma = e^2 L_0 (S/m),  seebeck = -(1/(e T)) L_0^{-1} L_1 (V/K, electron charge -e),
 *     kappa = (1/T)(L_2 - L_1 L_0^{-1} L_1) (W/(m K)),
 * no spin factor.  lattice: host, primitive vectors as rows (Angstrom), the cell of the R
 * coordinates of set_hamiltonian.  Outputs: host row-major 3 x 3.  Degenerate bands use
 * the diagonal velocity elements of the eigenvectors returned by the eigensolver. */
int phoebe_gpu_transport_rta(phoebe_gpu_ctx* ctx, const phoebe_gpu_rta_params* params, const double lattice[9],
                             double sigma[9], double seebeck[9], double kappa[9]);

/* ------------------------------------------------------------------------------------------
 * Importance-sampled q sums with a learned proposal.  The paper has no counterpart: Eq. 29
 * sums every q of the grid.  Write c_nk(q) for N_q times the q term of Eq. 29, so that
 * Gamma_nk = (1/N_q) sum_q c_nk(q).  The shell factor of a state is the bracket of Eq. 29 with
 * |g|^2 replaced by 1/(hbar w_q nu), summed over final bands and live modes (delta = the
 * truncated Gaussian of Eq. 61 without its normalisation):
 *     phi_nk(q) = sum_{m' nu} [(n + 1 - f_m'k+q) D(eps_nk - w - eps_m'k+q) + (n + f) D(eps_nk + w - ...)] / w;
 * it is zero exactly where every term of c_nk(q) is cut, so it vanishes wherever c does.
 * With params->sampler = PHOEBE_SAMPLER_LEARNED, linewidths_rta draws, per initial k,
 * S = ceil(sample_fraction * N_q) q points i.i.d. from
 *     p_k(q) = (1 - alpha) mean_n softmax_q (z_nk(q) + log phi_nk(q)) + alpha mean_n phi_nk(q) / sum_q phi_nk,
 * the means over the active bands n of k with some phi > 0 (1/N_q when there is none)
 * (inverse CDF in q-index order, FP64, Philox4x32-10 uniforms: draw j of k-grid index k uses
 * counter (j, k, 0x4953, 0), key (seed low word, seed high word), u = ((x1 << 32 | x0) >> 11) 2^-53)
 * and returns the unbiased estimate
 *     Gamma^_nk = (1/S) sum_j c_nk(q_j) / (N_q p_k(q_j)),
 * then averages degenerate bands as the full sum does.  PHOEBE_SAMPLER_SHELL uses
 * p_k = mean_n phi_nk / sum_q phi_nk, PHOEBE_SAMPLER_UNIFORM p_k = 1/N_q (neither needs the network).
 * All three need a tensor-core precision (1..6) and (nw, 3na) in
 * {(8,6), (2,3), (1,3)} with N_Rp * 3na * nw * 8 bytes <= 200 KB.
 * The network z = MLP(x), x = (q~, eps_nk - mu, v_nk): q~ is q wrapped into [-1/2, 1/2) per
 * axis, v_nk = <n| sum_R w_R i R e^{ik.R} H(R) |n> = (1/2 pi) d eps_nk / dk (eV, crystal axes);
 * 7 -> 128 -> 128 -> 128 -> 1 with SiLU after each hidden layer.  The context keeps FP32
 * master parameters; every evaluation uses them rounded to BF16 (ties to even), with FP32
 * activations and accumulation.  Parameter blob (float32, PHOEBE_GPU_MLP_NPARAM numbers):
 *     W1[128][7], b1[128], W2[128][128], b2[128], W3[128][128], b3[128], w4[128], b4.
 * ------------------------------------------------------------------------------------------ */
#define PHOEBE_GPU_MLP_NPARAM 34177

/* Seeded initialisation: weights uniform in +-1/sqrt(fan_in), biases 0; resets the optimiser. */
int phoebe_gpu_sampler_init(phoebe_gpu_ctx* ctx, uint64_t seed);
/* Set / read the FP32 master parameters (host blob of n = PHOEBE_GPU_MLP_NPARAM floats). */
int phoebe_gpu_sampler_load(phoebe_gpu_ctx* ctx, const float* params, int64_t n);
int phoebe_gpu_sampler_save(phoebe_gpu_ctx* ctx, float* params, int64_t n);

typedef struct {
  int epochs;                /* passes over the training states (default 60) */
  int states_per_step;       /* states per Adam step (default 64) */
  double lr, beta1, beta2, eps;  /* Adam (defaults 3e-3, 0.9, 0.999, 1e-8) */
  uint64_t seed;             /* order of the states in each epoch */
  int reserved[4];           /* must be zero */
} phoebe_gpu_train_opts;
void phoebe_gpu_train_opts_default(phoebe_gpu_train_opts* o);

/* Train the network on one full-grid run: computes c_nk(q) for every active state of `grid`
 * (its sampler field is ignored; its precision must be 1..6) and minimises, with Adam, the
 * mean over states of the cross entropy between t(q) = c_nk(q) / sum_q c_nk(q) and
 * softmax_q (z_nk(q) + log phi_nk(q)).  States with sum_q c = 0 are skipped.  loss_per_epoch (host, `epochs`
 * doubles, may be NULL) receives the mean loss of each epoch.  Needs init or load first. */
int phoebe_gpu_sampler_train(phoebe_gpu_ctx* ctx, const phoebe_gpu_rta_params* grid,
                             const phoebe_gpu_train_opts* opts, double* loss_per_epoch);

/* c_nk(q) for every active state and every q (host float [n_states][N_q], q in grid-index order),
 * the state features (host float [n_states][4]: eps - mu, v[3]; may be NULL) and log phi_nk(q)
 * (host float [n_states][N_q], -inf where phi = 0; may be NULL).  Two-call pattern as
 * linewidths_rta; precision must be 1..6. */
int phoebe_gpu_q_contributions(phoebe_gpu_ctx* ctx, const phoebe_gpu_rta_params* params, int* n_states,
                               int32_t* k_index, int32_t* band, float* c, float* features, float* log_shell);

/* The network and its training loss on explicit rows, for checking the kernels.
 *   x       host float [n_rows][7]
 *   group_off  host int64 [n_groups + 1] row offsets of the softmax groups (0 = first, n_rows = last)
 *   target  host float [n_rows] non-negative, or NULL (then only logits are computed)
 *   log_prior  host float [n_rows] additive log weights of the softmax (-inf allowed where the
 *              target is 0), or NULL (0)
 *   logits  host float [n_rows] or NULL (the network's z, without the prior)
 *   loss    mean over groups of -sum t log softmax(z + prior), t = target / its group sum (or NULL)
 *   grad    host float [PHOEBE_GPU_MLP_NPARAM] dloss/dparameters at the BF16-rounded values (or NULL) */
int phoebe_gpu_mlp_loss_grad(phoebe_gpu_ctx* ctx, int64_t n_rows, const float* x, int n_groups,
                             const int64_t* group_off, const float* target, const float* log_prior, float* logits,
                             double* loss, float* grad);

/* Network scores z for n_states feature rows (host float [n_states][4]: eps - mu, v[3]) over
 * every q of the grid nq (host float output [n_states][N_q], q in grid-index order).
 * tensor_cores = 1: the tcgen05 inference kernel the learned sampler uses (all three hidden
 * layers as MMAs with FP16 operands, the inputs rounded to FP16, FP32 accumulation, SiLU from
 * tanh.approx.f16x2; sm_10x only); 0: the CUDA-core forward pass of the training kernels (FP32
 * activations).  With profiling on, stats.sampler_ms holds the device time of the scoring. */
int phoebe_gpu_mlp_scores(phoebe_gpu_ctx* ctx, int n_states, const float* features, const int32_t nq[3],
                          int tensor_cores, float* z);

/* The uniforms u_j, j < n, of the draws for k-grid index k (as described above), host double [n]. */
int phoebe_gpu_is_uniforms(phoebe_gpu_ctx* ctx, uint64_t seed, int32_t k, int64_t n, double* u);

/* ------------------------------------------------------------------------------------------
 * Many materials in one call.  The paper has no counterpart (it treats one crystal per run).
 * Each item names a context holding one material (set_* done; all contexts on one device)
 * and its parameters (precision 1..6, sampler FULL; distinct contexts).  Phase 1 runs, per
 * material on its own context and stream, the grid band structure, phonons, window, stage 1
 * and the stage-2 operands, and records the material's stage-2 launches (with plan_threads > 1,
 * several materials at once on host threads); with autotune on, the tile width
 * (128 or 256 columns) and the K blocks per TMEM partial (1, 2 or 4) of its stage-2 GEMM are
 * chosen by timing each candidate once on the material's first q chunk; the context keeps the
 * choice per GEMM problem, and later batch calls with the same problem reuse it untimed.  Phase 2 captures
 * the recorded launches of all materials into one CUDA graph (materials spread round-robin
 * over n_streams parallel branches) and launches it once; items[0].ctx keeps the executable
 * graph, and a later call whose graph has the same shape updates it in place instead of
 * instantiating a new one (the kept graph is freed with that context).  Phase 3 averages degenerate
 * bands and writes each item's host outputs as linewidths_rta does.  Every shape uses the
 * stage 2 that writes G to HBM (the fused epilogue is not used in a batch); all of a
 * material's active states form one batch, so its operands must fit in device memory.
 * Two-call pattern: if any gamma_eV is NULL, only every n_states is written. */
typedef struct {
  phoebe_gpu_ctx* ctx;                  /* the material */
  const phoebe_gpu_rta_params* params;
  int n_states;                         /* in: output capacity; out: active states */
  int32_t* k_index;                     /* host outputs (may be NULL) */
  int32_t* band;
  double* gamma_eV;
  int tile_n, tile_kb;                  /* out: stage-2 tile columns and K blocks per partial used */
} phoebe_gpu_batch_item;

typedef struct {
  int autotune;              /* 1: time the tile candidates per material, once per context and
                                GEMM problem (default 1) */
  int n_streams;             /* parallel branches of the graph, 1..64 (default 4) */
  int64_t g_chunk_bytes;     /* stage-2 result buffer per material and q chunk (default 128 MiB) */
  double plan_ms;            /* out: phase 1 wall time (including the autotuner) */
  double graph_ms;           /* out: device time of the graph launch (every material's stage 2) */
  double finish_ms;          /* out: phase 3 wall time */
  int64_t graph_nodes;       /* out: nodes of the captured graph */
  int64_t recorded_launches; /* out: recorded stage-2 chunks (each a GEMM and an epilogue launch) */
  int plan_threads;          /* host threads of phase 1, each planning one material at a time on the
                                material's own stream, so that materials overlap on the GPU
                                (0 or 1 = one material after the other, the default; at most 64) */
  int graph_reused;          /* out: 1 if the executable graph of an earlier batch call (kept on
                                items[0].ctx) was updated in place instead of instantiated anew */
  int reserved[2];           /* must be zero */
} phoebe_gpu_batch_opts;

void phoebe_gpu_batch_opts_default(phoebe_gpu_batch_opts* o);
int phoebe_gpu_linewidths_rta_batch(phoebe_gpu_batch_item* items, int n, phoebe_gpu_batch_opts* opts);

/* Allocation-free band energies at explicit k points.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory -- host
 * programs sharing the GPU with a framework that has already reserved nearly all of
 * it for its own pool (cudaMalloc would fail), and latency-sensitive callers that
 * cannot accept the device-wide synchronisation cudaMalloc/cudaFree may imply.
 * It forms the Wannier sum H_k = sum_R w_R e^{ik.R} H(R) at each point and solves the
 * Hermitian eigenproblem of H_k (energies ascending, eigenvectors as columns) with the
 * same kernels as the grid path; it needs no context and allocates nothing: its only
 * scratch is a static 16 MiB device array that every GPU loading the library holds
 * until exit.
 *   nw, n_R      as for set_hamiltonian (nw <= 32)
 *   R, w, H      DEVICE arrays: n_R x 3 int32, n_R weights (not NULL), n_R x nw x nw
 *                complex (interleaved doubles), caller-owned
 *   n_k, k       n_k points, DEVICE array n_k x 3 crystal coordinates
 *   eps          DEVICE output n_k x nw, ascending
 *   U            DEVICE output n_k x nw x nw complex (columns = eigenvectors) or NULL
 *   cuda_stream  cudaStream_t of the work (NULL = default stream); the call returns
 *                after the stream has finished it.
 * Returns PHOEBE_GPU_ERR_NOMEM without launching anything when 2 * n_k * nw^2 * 16
 * bytes exceed the 16 MiB scratch, PHOEBE_GPU_ERR_ARG for bad sizes or NULL
 * pointers, PHOEBE_GPU_ERR_NOTCONVERGED if an eigensolve hit its QR step cap.
 * The first call on each device looks up the scratch address on the current device
 * (one-time set-up); make that first call before any stream capture begins.  Every
 * call reads its convergence word back and synchronises the stream, so a call on a
 * stream that is being captured returns PHOEBE_GPU_ERR_ARG before enqueuing anything
 * (the capture is left intact).  All calls on a device share the one scratch array:
 * calls that overlap on the GPU (other streams, other host threads) race on it. */
int phoebe_gpu_bands_noalloc(int nw, int n_R, const int32_t* R, const double* w, const double* H, int n_k,
                             const double* k, double* eps, double* U, void* cuda_stream);

/* Check of the bounded device waits of the pipeline kernels: one block waits on an mbarrier
 * phase that its producer publishes only when `publish` is non-zero.  Unpublished, the wait
 * gives up after limit_us microseconds (1..1e7) and the call returns PHOEBE_GPU_ERR_TIMEOUT;
 * the context stays usable.  Published, it returns PHOEBE_GPU_OK.  The paper has no
 * counterpart. */
int phoebe_gpu_selftest_wait(phoebe_gpu_ctx* ctx, int publish, int64_t limit_us);

/* Measured FP32 FMA rate of the device (the denominator of the CUDA-core roofline): 8 blocks of
 * 256 threads per SM, each thread 8 independent chains of 2^14 dependent FMAs; the fastest of three
 * timed launches after a warm-up, by CUDA events on the context's stream.  tflops (host, required)
 * = 2 flop x FMAs / time; ms (host, may be NULL) = that launch's time.  The paper has no
 * counterpart. */
int phoebe_gpu_selftest_fp32_rate(phoebe_gpu_ctx* ctx, double* tflops, double* ms);

/* Physical constants compiled into the library: out[0] = k_B (eV/K),
 * out[1] = hbar*sqrt(eV/(A^2 amu)) (eV), out[2] = hbar^2/(amu eV A^2).  Needs no GPU. */
void phoebe_gpu_constants(double out[3]);
/* Library version string.  Needs no GPU. */
const char* phoebe_gpu_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PHOEBE_GPU_H */
