// Orchestration of the linewidth path (grid band structure -> window ->
// stage 1 -> stage 2 -> rotations -> delta accumulation -> degenerate
// averaging) and of the explicit-pair coupling path.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pipeline.h"
#include "dft.h"
#include "tc.h"

namespace phx {

static int launch_check(phoebe_gpu_ctx* c, int n) {
  c->launches += n;
  CK(c, cudaGetLastError());
  return PHOEBE_GPU_OK;
}

static int electron_points(phoebe_gpu_ctx* c, const double* kdev, int64_t P, const char* tag, double** eps,
                           cplx** U) {
  int nw = c->nw, E = nw * nw, st;
  std::string t(tag);
  cplx* A = (cplx*)ensure(c, (t + "_A").c_str(), sizeof(cplx) * P * E, &st);
  if (!A) return st;
  cplx* V = (cplx*)ensure(c, (t + "_V").c_str(), sizeof(cplx) * P * E, &st);
  if (!V) return st;
  double* e = (double*)ensure(c, (t + "_eps").c_str(), sizeof(double) * P * nw, &st);
  if (!e) return st;
  cplx* u = (cplx*)ensure(c, (t + "_U").c_str(), sizeof(cplx) * P * E, &st);
  if (!u) return st;
  int* status = (int*)ensure(c, "status", 64, &st);
  if (!status) return st;
  CK(c, cudaMemsetAsync(status, 0, 64, c->stream));
  dim3 g((unsigned)((P + 127) / 128), (unsigned)E);
  k_fourier_points_c<<<g, 128, 0, c->stream>>>((const cplx*)c->bufs["H"].p, (const int*)c->bufs["RH"].p,
                                                 (const double*)c->bufs["wH"].p, c->nRH, E, kdev, P, A);
  if (eigh_launch(c->stream, A, V, nw, P, e, u, status)) return fail(c, PHOEBE_GPU_ERR_CUDA, "eigensolver launch failed");
  TRY(launch_check(c, 2));
  int hs = 0;
  CK(c, cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (hs) return fail(c, PHOEBE_GPU_ERR_NOTCONVERGED, "eigensolve of H(k) did not converge");
  *eps = e;
  *U = u;
  return PHOEBE_GPU_OK;
}

int interpolate_pairs(phoebe_gpu_ctx* c, int n_pairs, const double* k, const double* q, int precision,
                      double* g2, double* eps_k, double* eps_kq, double* omega_q) {
  c->launches = 0;
  if (n_pairs < 1 || !k || !q) return fail(c, PHOEBE_GPU_ERR_ARG, "interpolate_couplings: n_pairs < 1 or NULL k/q");
  if (precision < PHOEBE_PREC_FP64 || precision > PHOEBE_PREC_BF16X3)
    return fail(c, PHOEBE_GPU_ERR_ARG, "interpolate_couplings: unknown precision %d", precision);
  if (precision != PHOEBE_PREC_FP64)
    return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "interpolate_couplings: only PHOEBE_PREC_FP64 is implemented");
  if (!c->have_H || !c->have_Phi || !c->have_g)
    return fail(c, PHOEBE_GPU_ERR_ORDER, "interpolate_couplings needs all three set_* calls first");
  if (c->g_nw != c->nw || c->g_na != c->na)
    return fail(c, PHOEBE_GPU_ERR_SHAPE, "couplings were set for nw=%d, na=%d but H/Phi now have nw=%d, na=%d",
                c->g_nw, c->g_na, c->nw, c->na);
  const int nw = c->nw, nm = 3 * c->na;
  std::vector<double> kq(3 * (size_t)n_pairs);
  for (size_t i = 0; i < kq.size(); ++i) kq[i] = k[i] + q[i];
  void *dk, *dq, *dkq;
  TRY(upload(c, "pair_k", k, sizeof(double) * 3 * n_pairs, &dk));
  TRY(upload(c, "pair_q", q, sizeof(double) * 3 * n_pairs, &dq));
  TRY(upload(c, "pair_kq", kq.data(), sizeof(double) * 3 * n_pairs, &dkq));
  double *e0, *e1;
  cplx *U0, *U1;
  TRY(electron_points(c, (const double*)dk, n_pairs, "pk", &e0, &U0));
  TRY(electron_points(c, (const double*)dkq, n_pairs, "pkq", &e1, &U1));
  double *om, *nb;
  cplx* Zq;
  int dummy[3] = {1, 1, 1};
  TRY(phonon_modes(c, dummy, (const double*)dq, n_pairs, 300.0, 1e-4, &om, &nb, &Zq, "php"));
  if (g2) {
    const int64_t C = (int64_t)c->nRp * nw * nw * nm;
    const int PC = (int)std::max<int64_t>(1, std::min<int64_t>(n_pairs, (int64_t)(1ll << 30) / (C * 16)));
    int st;
    cplx* Pe = (cplx*)ensure(c, "pair_Pe", sizeof(cplx) * PC * c->nRe, &st);
    if (!Pe) return st;
    cplx* X = (cplx*)ensure(c, "pair_X", sizeof(cplx) * PC * C, &st);
    if (!X) return st;
    cplx* G = (cplx*)ensure(c, "pair_G", sizeof(cplx) * PC * nw * nw * nm, &st);
    if (!G) return st;
    double* out = (double*)ensure(c, "pair_g2", sizeof(double) * (size_t)n_pairs * nw * nw * nm, &st);
    if (!out) return st;
    for (int p0 = 0; p0 < n_pairs; p0 += PC) {
      int pc = std::min(PC, n_pairs - p0);
      int64_t nt = (int64_t)pc * c->nRe;
      k_phase_table_points<<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(
          Pe, (const double*)dk + 3 * p0, pc, (const int*)c->bufs["Re"].p, (const double*)c->bufs["we"].p, c->nRe);
      launch_zgemm(c->stream, pc, C, c->nRe, Pe, c->nRe, (const cplx*)c->bufs["g"].p, C, X, C);
      int64_t ng = (int64_t)pc * nw * nw * nm;
      k_pairs_stage2<<<(unsigned)((ng + 127) / 128), 128, 0, c->stream>>>(
          X, pc, (const double*)dq + 3 * p0, (const int*)c->bufs["Rp"].p, (const double*)c->bufs["wp"].p, c->nRp,
          nw, nm, G);
      int64_t nr = (int64_t)pc * nw * nw;
      k_pairs_rotate<<<(unsigned)((nr + 127) / 128), 128, 0, c->stream>>>(
          G, pc, U0 + (int64_t)p0 * nw * nw, U1 + (int64_t)p0 * nw * nw, Zq + (int64_t)p0 * nm * nm, nw, nm,
          out + (int64_t)p0 * nw * nw * nm);
      TRY(launch_check(c, 4));
    }
    CK(c, cudaMemcpyAsync(g2, out, sizeof(double) * (size_t)n_pairs * nw * nw * nm, cudaMemcpyDeviceToHost,
                          c->stream));
  }
  if (eps_k) CK(c, cudaMemcpyAsync(eps_k, e0, sizeof(double) * n_pairs * nw, cudaMemcpyDeviceToHost, c->stream));
  if (eps_kq) CK(c, cudaMemcpyAsync(eps_kq, e1, sizeof(double) * n_pairs * nw, cudaMemcpyDeviceToHost, c->stream));
  if (omega_q) CK(c, cudaMemcpyAsync(omega_q, om, sizeof(double) * n_pairs * nm, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return PHOEBE_GPU_OK;
}

// ------------------------------------------------------------------ linewidths

static int check_params(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, GridMap* gm) {
  if (!p) return fail(c, PHOEBE_GPU_ERR_ARG, "params is NULL");
  for (int i = 0; i < 3; ++i) {
    if (p->nk[i] < 1 || p->nq[i] < 1 || p->nk[i] > 4096 || p->nq[i] > 4096)
      return fail(c, PHOEBE_GPU_ERR_ARG, "grid sizes must be in 1..4096");
    int a = p->nk[i], b = p->nq[i];
    int hi = a > b ? a : b, lo = a > b ? b : a;
    if (hi % lo != 0)
      return fail(c, PHOEBE_GPU_ERR_GRID, "k grid %d and q grid %d along axis %d are not commensurate", a, b, i);
    gm->nk[i] = a;
    gm->nq[i] = b;
    gm->nf[i] = hi;
    gm->sk[i] = hi / a;
    gm->sq[i] = hi / b;
  }
  if (!(p->T_K > 0.0)) return fail(c, PHOEBE_GPU_ERR_ARG, "T_K must be > 0");
  if (!(p->sigma_eV > 0.0)) return fail(c, PHOEBE_GPU_ERR_ARG, "sigma_eV must be > 0");
  if (!(p->delta_cut_sigmas > 0.0)) return fail(c, PHOEBE_GPU_ERR_ARG, "delta_cut_sigmas must be > 0");
  if (!(p->omega_cut_eV >= 0.0)) return fail(c, PHOEBE_GPU_ERR_ARG, "omega_cut_eV must be >= 0");
  if (!(p->degen_tol_eV >= 0.0)) return fail(c, PHOEBE_GPU_ERR_ARG, "degen_tol_eV must be >= 0");
  if (p->precision < PHOEBE_PREC_FP64 || p->precision > PHOEBE_PREC_FP64_DFT)
    return fail(c, PHOEBE_GPU_ERR_ARG, "unknown precision %d", p->precision);
  if (p->reserved1 != 0) return fail(c, PHOEBE_GPU_ERR_ARG, "reserved fields must be zero");
  if (c->have_polar) {
    if (p->precision != PHOEBE_PREC_FP32_DFT || p->sampler != PHOEBE_SAMPLER_FULL || p->smearing != 0 ||
        c->prate_acc)
      return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED,
                  "the polar long-range term is evaluated by the grid-DFT linewidths (precision 7, full q sum, "
                  "fixed smearing)");
    if (!c->have_lattice) return fail(c, PHOEBE_GPU_ERR_ORDER, "the polar term needs set_lattice first");
    if ((int)c->zstar.size() != 9 * c->na)
      return fail(c, PHOEBE_GPU_ERR_SHAPE, "Born charges were set for another atom count");
  }
  if (p->window_final != 0 && p->window_final != 1) return fail(c, PHOEBE_GPU_ERR_ARG, "window_final must be 0 or 1");
  if (p->window_final == 1 && (p->precision != PHOEBE_PREC_FP32_DFT || p->sampler != PHOEBE_SAMPLER_FULL))
    return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED,
                "final-state windows are evaluated by the grid-DFT stage 2 (precision 7, full q sum)");
  if (p->smearing != 0 && p->smearing != 1) return fail(c, PHOEBE_GPU_ERR_ARG, "smearing must be 0 or 1");
  if (p->smearing == 1) {
    if (!(p->sigma_min_eV > 0.0)) return fail(c, PHOEBE_GPU_ERR_ARG, "sigma_min_eV must be > 0");
    if (p->precision != PHOEBE_PREC_FP32_DFT || p->sampler != PHOEBE_SAMPLER_FULL)
      return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED,
                  "adaptive smearing is evaluated by the grid-DFT stage 2 (precision 7, full q sum)");
    if (!c->have_lattice) return fail(c, PHOEBE_GPU_ERR_ORDER, "adaptive smearing needs set_lattice first");
    if (c->prate_acc)
      return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "phonon-electron rates use the fixed Gaussian width");
  }
  if (!(p->population_delta >= 0.0 && p->population_delta < 0.25))
    return fail(c, PHOEBE_GPU_ERR_ARG, "population_delta must be in [0, 0.25)");
  if (p->sampler_fp32_network != 0 && p->sampler_fp32_network != 1)
    return fail(c, PHOEBE_GPU_ERR_ARG, "sampler_fp32_network must be 0 or 1");
  if (p->sampler < PHOEBE_SAMPLER_FULL || p->sampler > PHOEBE_SAMPLER_SHELL)
    return fail(c, PHOEBE_GPU_ERR_ARG, "unknown sampler %d", p->sampler);
  if (p->sampler != PHOEBE_SAMPLER_FULL) {
    if (!(p->sample_fraction > 0.0 && p->sample_fraction <= 1.0))
      return fail(c, PHOEBE_GPU_ERR_ARG, "sample_fraction must be in (0, 1]");
    if (p->sampler == PHOEBE_SAMPLER_LEARNED && !(p->mix_alpha > 0.0 && p->mix_alpha <= 1.0))
      return fail(c, PHOEBE_GPU_ERR_ARG, "mix_alpha must be in (0, 1]");
    if (p->precision == PHOEBE_PREC_FP64)
      return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "sampled q sums need a tensor-core precision (1..6)");
    if (p->sampler == PHOEBE_SAMPLER_LEARNED && !c->have_mlp)
      return fail(c, PHOEBE_GPU_ERR_ORDER, "the learned sampler needs sampler_init/load/train first");
  }
  if (p->max_batch_states < 0) return fail(c, PHOEBE_GPU_ERR_ARG, "max_batch_states must be >= 0");
  int64_t Nk = (int64_t)p->nk[0] * p->nk[1] * p->nk[2];
  if (p->n_k_subset < 0) return fail(c, PHOEBE_GPU_ERR_ARG, "n_k_subset must be >= 0");
  if (p->n_k_subset > 0) {
    if (!p->k_subset) return fail(c, PHOEBE_GPU_ERR_ARG, "k_subset is NULL");
    for (int i = 0; i < p->n_k_subset; ++i) {
      if (p->k_subset[i] < 0 || p->k_subset[i] >= Nk)
        return fail(c, PHOEBE_GPU_ERR_GRID, "k_subset[%d]=%d outside the k grid", i, p->k_subset[i]);
      if (i > 0 && p->k_subset[i] <= p->k_subset[i - 1])
        return fail(c, PHOEBE_GPU_ERR_GRID, "k_subset must be strictly ascending");
    }
  }
  return PHOEBE_GPU_OK;
}

static int run_fp64(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, const GridMap& gm, int64_t ns,
                    const std::vector<int>& hk, const int* st_k, const int* st_b, const double* epsF,
                    const cplx* UF, const double* fF, const double* omega, const double* nB, const cplx* Zq,
                    double* raw) {
  const int nw = c->nw, nm = 3 * c->na, nRe = c->nRe, nRp = c->nRp;
  const int64_t Nq = (int64_t)gm.nq[0] * gm.nq[1] * gm.nq[2];
  const int64_t C = (int64_t)nRp * nw * nw * nm;
  int st;
  // q phase table P[q][Rp] (k independent)
  GridPhase gq = make_phase(gm.nq), gk = make_phase(gm.nk);
  cplx *cis_q, *cis_k;
  TRY(cis_table(c, gq, "cis_q", &cis_q));
  TRY(cis_table(c, gk, "cis_k", &cis_k));
  Timer t;
  t.begin(c);
  cplx* Pq = (cplx*)ensure(c, "Pq", sizeof(cplx) * Nq * nRp, &st);
  if (!Pq) return st;
  k_phase_table_grid<<<(unsigned)((Nq * nRp + 255) / 256), 256, 0, c->stream>>>(
      Pq, nullptr, Nq, (const int*)c->bufs["Rp"].p, (const double*)c->bufs["wp"].p, nRp, gq, cis_q);
  TRY(launch_check(c, 1));
  t.end(c, &c->stats.stage1_ms);

  // largest phonon energy: bands farther than omega_max + cut sigma from eps_nk have every term cut
  unsigned long long* dmax = (unsigned long long*)ensure(c, "fp64_wmax", 64, &st);
  if (!dmax) return st;
  CK(c, cudaMemsetAsync(dmax, 0, 64, c->stream));
  k_absmax_f64<<<64, 256, 0, c->stream>>>(omega, Nq * nm, dmax);
  TRY(launch_check(c, 1));
  unsigned long long ombits = 0;
  CK(c, cudaMemcpyAsync(&ombits, dmax, sizeof(ombits), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  double omega_max;
  memcpy(&omega_max, &ombits, sizeof(double));
  int S_max = p->max_batch_states > 0 ? p->max_batch_states : 64;
  const double pref = 2.0 * kPi / (double)Nq;
  const size_t budget = (size_t)4 << 30;
  int64_t i0 = 0;
  std::vector<int> kb_list, st_kb;
  while (i0 < ns) {
    int64_t i1 = std::min<int64_t>(ns, i0 + S_max);
    while (i1 < ns && hk[i1] == hk[i1 - 1]) ++i1;  // do not split a k across batches
    int S = (int)(i1 - i0);
    kb_list.clear();
    st_kb.assign(S, 0);
    for (int64_t s = i0; s < i1; ++s) {
      if (kb_list.empty() || kb_list.back() != hk[s]) kb_list.push_back(hk[s]);
      st_kb[s - i0] = (int)kb_list.size() - 1;
    }
    int nkb = (int)kb_list.size();
    void *d_kb, *d_stkb;
    TRY(upload(c, "batch_k", kb_list.data(), sizeof(int) * nkb, &d_kb));
    TRY(upload(c, "batch_stkb", st_kb.data(), sizeof(int) * S, &d_stkb));
    // stage 1
    t.begin(c);
    cplx* Pe = (cplx*)ensure(c, "Pe", sizeof(cplx) * nkb * nRe, &st);
    if (!Pe) return st;
    cplx* X = (cplx*)ensure(c, "X", sizeof(cplx) * nkb * C, &st);
    if (!X) return st;
    cplx* T = (cplx*)ensure(c, "T", sizeof(cplx) * (size_t)nRp * S * nw * nm, &st);
    if (!T) return st;
    k_phase_table_grid<<<(unsigned)(((int64_t)nkb * nRe + 255) / 256), 256, 0, c->stream>>>(
        Pe, (const int*)d_kb, nkb, (const int*)c->bufs["Re"].p, (const double*)c->bufs["we"].p, nRe, gk, cis_k);
    launch_zgemm(c->stream, nkb, C, nRe, Pe, nRe, (const cplx*)c->bufs["g"].p, C, X, C);
    int64_t ntp = (int64_t)nRp * S * nw * nm;
    k_tpack_fp64<<<(unsigned)((ntp + 127) / 128), 128, 0, c->stream>>>(X, C, (const int*)d_stkb, st_k + i0,
                                                                          st_b + i0, gm, UF, S, nRp, nw, nm, T);
    TRY(launch_check(c, 3));
    t.end(c, &c->stats.stage1_ms);
    // stage 2 over q chunks
    const int64_t N2 = (int64_t)S * nw * nm;
    int64_t Qc = std::max<int64_t>(1, std::min<int64_t>(Nq, (int64_t)(budget / (N2 * 24))));
    cplx* G = (cplx*)ensure(c, "G", sizeof(cplx) * Qc * N2, &st);
    if (!G) return st;
    double* g2 = (double*)ensure(c, "g2", sizeof(double) * Qc * N2, &st);
    if (!g2) return st;
    for (int64_t q0 = 0; q0 < Nq; q0 += Qc) {
      int64_t qc = std::min(Qc, Nq - q0);
      t.begin(c);
      launch_zgemm(c->stream, qc, N2, nRp, Pq + q0 * nRp, nRp, T, N2, G, N2);
      TRY(launch_check(c, 1));
      c->stats.stage2_launches++;
      t.end(c, &c->stats.stage2_ms);
      t.begin(c);
      dim3 gr((unsigned)((qc + 127) / 128), (unsigned)S);
      k_rotate_final_fp64<<<gr, 128, 0, c->stream>>>(G, S, qc, q0, st_k + i0, gm, UF, Zq, nw, nm, g2);
      TRY(launch_check(c, 1));
      t.end(c, &c->stats.rotate_ms);
      t.begin(c);
      unsigned bx = (unsigned)std::min<int64_t>((qc + 255) / 256, 64);
      k_delta_accumulate_fp64<<<dim3(bx, (unsigned)S), 256, 0, c->stream>>>(
          g2, S, qc, q0, st_k + i0, st_b + i0, i0, gm, epsF, fF, omega, nB, nw, nm, p->sigma_eV,
          p->delta_cut_sigmas, pref, (omega_max + p->delta_cut_sigmas * p->sigma_eV) * (1.0 + 1e-12), raw);
      TRY(launch_check(c, 1));
      t.end(c, &c->stats.delta_ms);
    }
    i0 = i1;
  }
  c->stats.pairs_executed = ns * Nq;
  c->stats.stage2_flops = 8.0 * (double)Nq * nRp * (double)ns * nw * nm;
  return PHOEBE_GPU_OK;
}

// Degenerate averaging (a12) of the raw accumulator into the outputs.
static int finish_outputs(phoebe_gpu_ctx* c, const GridMap& gm, int64_t ns, double degen_tol, int32_t* k_index,
                          int32_t* band, double* gamma, bool device_out) {
  int st;
  const int nw = c->nw;
  const double* raw = (const double*)c->bufs["gamma_raw"].p;
  const int* st_k = (const int*)c->bufs["st_k"].p;
  const int* st_b = (const int*)c->bufs["st_b"].p;
  const double* epsF = (const double*)c->bufs["epsF"].p;
  double* out = gamma;
  if (!device_out) {
    out = (double*)ensure(c, "gamma_out", sizeof(double) * ns, &st);
    if (!out) return st;
  }
  k_degenerate_average<<<(unsigned)((ns + 255) / 256), 256, 0, c->stream>>>(raw, st_k, st_b, ns, epsF, gm, nw,
                                                                            degen_tol, out);
  TRY(launch_check(c, 1));
  cudaMemcpyKind kind = device_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (!device_out) CK(c, cudaMemcpyAsync(gamma, out, sizeof(double) * ns, kind, c->stream));
  if (k_index) CK(c, cudaMemcpyAsync(k_index, st_k, sizeof(int) * ns, kind, c->stream));
  if (band) CK(c, cudaMemcpyAsync(band, st_b, sizeof(int) * ns, kind, c->stream));
  if (!device_out) CK(c, cudaStreamSynchronize(c->stream));
  return PHOEBE_GPU_OK;
}

namespace {
// Installs an importance-sampling request for one call when the parameters ask for one.
struct IsGuard {
  phoebe_gpu_ctx* c;
  IsRequest req;
  bool own = false;
  IsGuard(phoebe_gpu_ctx* ctx, const phoebe_gpu_rta_params* p) : c(ctx) {
    if (!c->isreq && p && p->sampler != PHOEBE_SAMPLER_FULL) {
      req.mode = 1;
      c->isreq = &req;
      own = true;
    }
  }
  ~IsGuard() {
    if (own) c->isreq = nullptr;
  }
};
}  // namespace

int linewidths(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, int* n_states, int32_t* k_index, int32_t* band,
               double* gamma, bool device_out) {
  c->launches = 0;
  memset(&c->stats, 0, sizeof(c->stats));
  if (!n_states) return fail(c, PHOEBE_GPU_ERR_ARG, "n_states is NULL");
  GridMap gm;
  TRY(check_params(c, p, &gm));
  IsGuard is_guard(c, p);
  if (c->isreq && p->precision == PHOEBE_PREC_FP64)
    return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "sampled q sums need a tensor-core precision (1..6)");
  if (!c->have_H || !c->have_Phi || !c->have_g)
    return fail(c, PHOEBE_GPU_ERR_ORDER, "linewidths_rta needs all three set_* calls first");
  if (c->g_nw != c->nw || c->g_na != c->na)
    return fail(c, PHOEBE_GPU_ERR_SHAPE, "couplings were set for nw=%d, na=%d but H/Phi now have nw=%d, na=%d",
                c->g_nw, c->g_na, c->nw, c->na);
  Timer total;
  total.begin(c);
  const int nw = c->nw, nm = 3 * c->na;
  const int64_t NF = (int64_t)gm.nf[0] * gm.nf[1] * gm.nf[2];
  const int64_t Nk = (int64_t)gm.nk[0] * gm.nk[1] * gm.nk[2];
  const int64_t Nq = (int64_t)gm.nq[0] * gm.nq[1] * gm.nq[2];
  int st;
  Timer t;
  // electrons on the fine grid (a1-a2)
  t.begin(c);
  double* epsF;
  cplx* UF;
  TRY(electron_grid(c, gm.nf, &epsF, &UF));
  double* fF = (double*)ensure(c, "fF", sizeof(double) * NF * nw, &st);
  if (!fF) return st;
  k_fermi<<<(unsigned)((NF * nw + 255) / 256), 256, 0, c->stream>>>(epsF, NF * nw, p->mu_eV, p->T_K, fF);
  TRY(launch_check(c, 1));
  t.end(c, &c->stats.bands_ms);
  // phonons on the q grid (a3-a5)
  t.begin(c);
  double *omega, *nB;
  cplx* Zq;
  TRY(phonon_modes(c, gm.nq, nullptr, Nq, p->T_K, p->omega_cut_eV, &omega, &nB, &Zq, "phq"));
  t.end(c, &c->stats.phonons_ms);
  // window (a6)
  t.begin(c);
  int64_t NC = p->n_k_subset > 0 ? p->n_k_subset : Nk;
  const int* kidx = nullptr;
  if (p->n_k_subset > 0) {
    void* d;
    TRY(upload(c, "k_subset", p->k_subset, sizeof(int32_t) * NC, &d));
    kidx = (const int*)d;
  }
  int* count = (int*)ensure(c, "win_count", sizeof(int) * NC, &st);
  if (!count) return st;
  int64_t* offset = (int64_t*)ensure(c, "win_off", sizeof(int64_t) * (NC + 1), &st);
  if (!offset) return st;
  double window = p->window_eV;
  const double kT = kBoltzmannEV * p->T_K;
  k_window_count<<<(unsigned)((NC + 255) / 256), 256, 0, c->stream>>>(epsF, kidx, NC, nw, gm, p->mu_eV, window, kT,
                                                                       p->population_delta, count);
  k_scan_single_block<<<1, 1024, 0, c->stream>>>(count, NC, offset);
  TRY(launch_check(c, 2));
  int64_t ns = 0;
  CK(c, cudaMemcpyAsync(&ns, offset + NC, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (!gamma) {
    *n_states = (int)ns;
    t.end(c, &c->stats.window_ms);
    return PHOEBE_GPU_OK;
  }
  if (*n_states < ns)
    return fail(c, PHOEBE_GPU_ERR_ARG, "output capacity %d is below the %lld active states", *n_states,
                (long long)ns);
  int* st_k = (int*)ensure(c, "st_k", sizeof(int) * (ns + 1), &st);
  if (!st_k) return st;
  int* st_b = (int*)ensure(c, "st_b", sizeof(int) * (ns + 1), &st);
  if (!st_b) return st;
  k_window_write<<<(unsigned)((NC + 255) / 256), 256, 0, c->stream>>>(epsF, kidx, NC, nw, gm, p->mu_eV, window, kT,
                                                                       p->population_delta, offset, st_k, st_b);
  TRY(launch_check(c, 1));
  t.end(c, &c->stats.window_ms);
  c->stats.n_states = ns;
  c->stats.n_q = Nq;
  c->stats.pairs_dense = ns * Nq;
  c->stats.couplings_dense = ns * Nq * nw * nm;
  *n_states = (int)ns;
  if (ns == 0) {
    total.end(c, &c->stats.total_ms);
    return PHOEBE_GPU_OK;
  }
  std::vector<int> hk(ns);
  CK(c, cudaMemcpyAsync(hk.data(), st_k, sizeof(int) * ns, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  int64_t nkd = 1;
  for (int64_t i = 1; i < ns; ++i) nkd += hk[i] != hk[i - 1];
  c->stats.n_k = nkd;
  double* raw = (double*)ensure(c, "gamma_raw", sizeof(double) * ns, &st);
  if (!raw) return st;
  CK(c, cudaMemsetAsync(raw, 0, sizeof(double) * ns, c->stream));
  if (c->defer && p->precision == PHOEBE_PREC_FP64)
    return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "batched linewidths need a tensor-core precision (1..6)");
  if (p->precision == PHOEBE_PREC_FP64) {
    TRY(run_fp64(c, p, gm, ns, hk, st_k, st_b, epsF, UF, fF, omega, nB, Zq, raw));
  } else {
    TRY(run_tc(c, p, gm, ns, hk, st_k, st_b, epsF, UF, fF, omega, nB, Zq, raw));
  }
  c->stats.couplings_executed = c->stats.pairs_executed * nw * nm;
  if (c->prate_acc) {  // phonon-electron rates accumulated by the grid-DFT stage 2
    const double Nk = (double)gm.nk[0] * gm.nk[1] * gm.nk[2];
    const double pref = 2.0 * kPi / (Nk * kSqrtPi * p->sigma_eV);
    if (prate_finish(c->stream, c->prate_acc, omega, nB, Nq, nm, pref, p->omega_cut_eV, p->degen_tol_eV,
                     c->prate_out)) {
      cudaGetLastError();
      return fail(c, PHOEBE_GPU_ERR_CUDA, "launch of the phonon-rate finish failed");
    }
    c->launches++;
  }
  if (c->defer) {  // stage 2 recorded, not run: finish later
    c->defer->ns = ns;
    c->defer->gm = gm;
    c->defer->degen_tol = p->degen_tol_eV;
    total.end(c, &c->stats.total_ms);
    c->stats.kernel_launches = c->launches;
    return PHOEBE_GPU_OK;
  }
  TRY(finish_outputs(c, gm, ns, p->degen_tol_eV, k_index, band, gamma, device_out));
  total.end(c, &c->stats.total_ms);
  c->stats.kernel_launches = c->launches;
  return PHOEBE_GPU_OK;
}

int linewidths_finish(phoebe_gpu_ctx* c, int32_t* k_index, int32_t* band, double* gamma, bool device_out) {
  if (!c->defer) return fail(c, PHOEBE_GPU_ERR_ORDER, "no deferred linewidth call to finish");
  if (c->defer->ns == 0) return PHOEBE_GPU_OK;
  return finish_outputs(c, c->defer->gm, c->defer->ns, c->defer->degen_tol, k_index, band, gamma, device_out);
}

}  // namespace phx
