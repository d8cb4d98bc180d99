// FP64 coupling interpolation and linewidth accumulation on CUDA cores.
//
// Stage 1 (Sec. 5.5, Eq. 71): X[k][Rp,m,n,sa] = sum_Re w_e e^{i k.Re} g[Re][Rp,m,n,sa]
//   as a complex GEMM of the k-batch phase table with g, followed by the
//   U_k rotation of n onto the active bands b (k_tpack_fp64), giving
//   T[Rp][s][m][sa] for the states s of the batch.
// Stage 2 (Eq. 70, the R_p sum): G[q][s,m,sa] = sum_Rp w_p e^{i q.Rp} T[Rp][s,m,sa]
//   as a complex GEMM of the q phase table with T.
// Final rotation (Eq. 13 with Eq. 7): g[m'][nu] = sum [U_{k+q}^dagger]_{m'm} G[m][sa] Z_q[sa][nu]
//   -> |g|^2 streamed to HBM as g2[s][m'][nu][q].
// Delta accumulation (Eq. 29 with Eq. 61): an HBM-streaming pass over g2.
#include "kernels.cuh"

namespace phx {

// P[i][r] = w_r e^{2 pi i k_i.R_r} for grid points pts[i] (grid indices) or all points.
__global__ void k_phase_table_grid(cplx* __restrict__ P, const int* __restrict__ pts, int64_t npts,
                                   const int* __restrict__ R, const double* __restrict__ w, int nR,
                                   GridPhase gp, const cplx* __restrict__ cis) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= npts * nR) return;
  int64_t i = t / nR;
  int r = (int)(t % nR);
  int64_t idx = pts ? pts[i] : i;
  int j[3];
  grid_coords(idx, gp.n, j);
  int Rv[3] = {R[3 * r], R[3 * r + 1], R[3 * r + 2]};
  cplx ph = cis[phase_index(j, Rv, gp.mult, gp.L)];
  P[t] = {ph.re * w[r], ph.im * w[r]};
}

// Same for arbitrary crystal-coordinate points.
__global__ void k_phase_table_points(cplx* __restrict__ P, const double* __restrict__ pts, int64_t npts,
                                     const int* __restrict__ R, const double* __restrict__ w, int nR) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= npts * nR) return;
  int64_t i = t / nR;
  int r = (int)(t % nR);
  double x = pts[3 * i] * R[3 * r] + pts[3 * i + 1] * R[3 * r + 1] + pts[3 * i + 2] * R[3 * r + 2];
  x -= floor(x);
  double s, c;
  sincospi(2.0 * x, &s, &c);
  P[t] = {c * w[r], s * w[r]};
}

// C[M x N] = A[M x K] B[K x N], complex FP64, row-major with leading dimensions.
// 64x64 output tile per 256-thread block, 4x4 outputs per thread (strided by 16
// so shared-memory reads are conflict-free), K staged 8 at a time.
constexpr int ZG_BM = 64, ZG_BN = 64, ZG_BK = 8;

__global__ void __launch_bounds__(256) k_zgemm(int64_t M, int64_t N, int K, const cplx* __restrict__ A,
                                               int64_t lda, const cplx* __restrict__ B, int64_t ldb,
                                               cplx* __restrict__ C, int64_t ldc) {
  __shared__ cplx As[ZG_BK][ZG_BM + 1];
  __shared__ cplx Bs[ZG_BK][ZG_BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.y * ZG_BM, n0 = (int64_t)blockIdx.x * ZG_BN;
  cplx acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = {0.0, 0.0};
  for (int k0 = 0; k0 < K; k0 += ZG_BK) {
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      int idx = tid + l * 256;
      int r = idx / ZG_BK, c = idx % ZG_BK;           // A tile: 64 rows x 8 cols
      int64_t gm = m0 + r;
      int gk = k0 + c;
      As[c][r] = (gm < M && gk < K) ? A[gm * lda + gk] : cplx{0.0, 0.0};
      int rb = idx / ZG_BN, cb = idx % ZG_BN;         // B tile: 8 rows x 64 cols
      int gkb = k0 + rb;
      int64_t gn = n0 + cb;
      Bs[rb][cb] = (gkb < K && gn < N) ? B[(int64_t)gkb * ldb + gn] : cplx{0.0, 0.0};
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < ZG_BK; ++kk) {
      cplx a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t gn = n0 + tx + 16 * j;
      if (gn < N) C[gm * ldc + gn] = acc[i][j];
    }
  }
}

void launch_zgemm(cudaStream_t s, int64_t M, int64_t N, int K, const cplx* A, int64_t lda, const cplx* B,
                  int64_t ldb, cplx* C, int64_t ldc) {
  dim3 grid((unsigned)((N + ZG_BN - 1) / ZG_BN), (unsigned)((M + ZG_BM - 1) / ZG_BM));
  k_zgemm<<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
}

// T[Rp][s][m][sa] = sum_n X[kb(s)][Rp][m][n][sa] U_k(s)[n][b(s)]   (Eq. 71's U_k rotation).
// st_kb[s] = row of the stage-1 output holding the state's k.
__global__ void k_tpack_fp64(const cplx* __restrict__ X, int64_t ldx, const int* __restrict__ st_kb,
                             const int* __restrict__ st_k, const int* __restrict__ st_b, GridMap gm,
                             const cplx* __restrict__ UF, int S, int nRp, int nw, int nm,
                             cplx* __restrict__ T) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t per_rp = (int64_t)S * nw * nm;
  if (t >= per_rp * nRp) return;
  int64_t rp = t / per_rp;
  int64_t rem = t % per_rp;
  int s = (int)(rem / (nw * nm));
  int m = (int)((rem / nm) % nw);
  int sa = (int)(rem % nm);
  const cplx* x = X + (int64_t)st_kb[s] * ldx + ((rp * nw + m) * nw) * nm + sa;
  const cplx* U = UF + gm.k_to_fine(st_k[s]) * nw * nw;
  int b = st_b[s];
  cplx acc = {0.0, 0.0};
  for (int n = 0; n < nw; ++n) cfma(acc, x[(int64_t)n * nm], U[n * nw + b]);
  T[t] = acc;
}

// |g|^2 of the states of a batch for the q chunk [q0, q0+Qc):
// g[m'][nu] = sum_m conj(U_{k+q}[m][m']) sum_sa G[q][s][m][sa] Z_q[sa][nu].
// Output g2[s][m'][nu][q - q0] (q fastest, so the delta pass streams it).
__global__ void k_rotate_final_fp64(const cplx* __restrict__ G, int S, int64_t Qc, int64_t q0,
                                    const int* __restrict__ st_k, GridMap gm, const cplx* __restrict__ UF,
                                    const cplx* __restrict__ Zq, int nw, int nm, double* __restrict__ g2) {
  int64_t ql = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int s = blockIdx.y;
  if (ql >= Qc) return;
  int64_t q = q0 + ql;
  int64_t kq = gm.kq_to_fine(st_k[s], q);
  const cplx* Gq = G + (ql * S + s) * (int64_t)nw * nm;
  const cplx* U = UF + kq * nw * nw;
  const cplx* Z = Zq + q * nm * nm;
  cplx t[kMaxNw];
  for (int nu = 0; nu < nm; ++nu) {
    for (int m = 0; m < nw; ++m) {
      cplx a = {0.0, 0.0};
      for (int sa = 0; sa < nm; ++sa) cfma(a, Gq[m * nm + sa], Z[sa * nm + nu]);
      t[m] = a;
    }
    for (int mp = 0; mp < nw; ++mp) {
      cplx a = {0.0, 0.0};
      for (int m = 0; m < nw; ++m) cfma_conja(a, U[m * nw + mp], t[m]);
      g2[(((int64_t)s * nw + mp) * nm + nu) * Qc + ql] = cabs2(a);
    }
  }
}

// Gamma_raw[s] += pref * sum_{q in chunk} sum_{m' nu} g2 * [(n+1-f) d(e - w - e') + (n+f) d(e + w - e')]
// with d the Gaussian of Eq. 61 truncated at cut*sigma.  A final band with |e - e'| >= reach =
// omega_max + cut*sigma has every term cut, so its |g|^2 is not read and costs no FP64 work; the
// other bands' terms are tested and weighted in FP64.  g2 columns are q (consecutive threads read
// consecutive q).
__global__ void __launch_bounds__(256) k_delta_accumulate_fp64(
    const double* __restrict__ g2, int S, int64_t Qc, int64_t q0, const int* __restrict__ st_k,
    const int* __restrict__ st_b, int64_t s_base, GridMap gm, const double* __restrict__ epsF,
    const double* __restrict__ fF, const double* __restrict__ omega, const double* __restrict__ nB, int nw,
    int nm, double sigma, double cut, double pref, double reach, double* __restrict__ gamma) {
  int s = blockIdx.y;
  int64_t kk = st_k[s];
  double e = epsF[gm.k_to_fine(kk) * nw + st_b[s]];
  double inv_s = 1.0 / sigma, norm = 1.0 / (kSqrtPi * sigma), xcut = cut * sigma;
  double acc = 0.0;
  for (int64_t ql = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ql < Qc;
       ql += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = q0 + ql;
    int64_t kq = gm.kq_to_fine(kk, q);
    for (int mp = 0; mp < nw; ++mp) {
      double ep = epsF[kq * nw + mp];
      if (!(fabs(e - ep) < reach)) continue;  // every Gaussian of this band is cut
      double f = fF[kq * nw + mp];
      const double* gv = g2 + ((int64_t)s * nw + mp) * nm * Qc + ql;
      for (int nu = 0; nu < nm; ++nu) {
        double w = omega[q * nm + nu];
        double n = nB[q * nm + nu];
        double x1 = e - w - ep, x2 = e + w - ep;
        double d = 0.0;
        if (fabs(x1) < xcut) d += (n + 1.0 - f) * exp(-(x1 * inv_s) * (x1 * inv_s));
        if (fabs(x2) < xcut) d += (n + f) * exp(-(x2 * inv_s) * (x2 * inv_s));
        if (d != 0.0) acc = fma(gv[(int64_t)nu * Qc], d, acc);
      }
    }
  }
  // block reduction
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(gamma + s_base + s, v * pref * norm);
  }
}

// out[s] = mean of raw over the active states at the same k with |eps - eps_s| < tol.
// States of one k are contiguous (k-then-band order).
__global__ void k_degenerate_average(const double* __restrict__ raw, const int* __restrict__ st_k,
                                     const int* __restrict__ st_b, int64_t NS, const double* __restrict__ epsF,
                                     GridMap gm, int nw, double tol, double* __restrict__ out) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= NS) return;
  int k = st_k[s];
  int64_t f = gm.k_to_fine(k);
  double e = epsF[f * nw + st_b[s]];
  int64_t lo = s, hi = s;
  while (lo > 0 && st_k[lo - 1] == k) --lo;
  while (hi + 1 < NS && st_k[hi + 1] == k) ++hi;
  double sum = 0.0;
  int cnt = 0;
  for (int64_t j = lo; j <= hi; ++j) {
    if (fabs(epsF[f * nw + st_b[j]] - e) < tol) {
      sum += raw[j];
      ++cnt;
    }
  }
  out[s] = sum / cnt;
}

// Explicit pairs, stage 2: G[p][m][n][sa] = sum_Rp w_p e^{i q_p.Rp} X[p][Rp][m][n][sa].
__global__ void k_pairs_stage2(const cplx* __restrict__ X, int npairs, const double* __restrict__ q,
                               const int* __restrict__ Rp, const double* __restrict__ wp, int nRp, int nw,
                               int nm, cplx* __restrict__ G) {
  int64_t per = (int64_t)nw * nw * nm;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= per * npairs) return;
  int p = (int)(t / per);
  int64_t e = t % per;
  cplx acc = {0.0, 0.0};
  for (int r = 0; r < nRp; ++r) {
    double x = q[3 * p] * Rp[3 * r] + q[3 * p + 1] * Rp[3 * r + 1] + q[3 * p + 2] * Rp[3 * r + 2];
    x -= floor(x);
    double sn, cs;
    sincospi(2.0 * x, &sn, &cs);
    cfma(acc, {cs * wp[r], sn * wp[r]}, X[((int64_t)p * nRp + r) * per + e]);
  }
  G[t] = acc;
}

// Explicit pairs, final rotation: g2[p][m'][n][nu] = |sum U_{k+q}^dagger G U_k Z|^2 with
// G[p][m][n'][sa] not yet rotated on n' (stage 1 without U_k for pairs).
__global__ void k_pairs_rotate(const cplx* __restrict__ G, int npairs, const cplx* __restrict__ Uk,
                               const cplx* __restrict__ Ukq, const cplx* __restrict__ Zq, int nw, int nm,
                               double* __restrict__ g2) {
  int64_t per = (int64_t)nw * nw;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= per * npairs) return;
  int p = (int)(t / per);
  int mp = (int)((t % per) / nw), n = (int)(t % nw);
  const cplx* Gp = G + (int64_t)p * nw * nw * nm;
  const cplx* U1 = Ukq + (int64_t)p * nw * nw;
  const cplx* U0 = Uk + (int64_t)p * nw * nw;
  const cplx* Z = Zq + (int64_t)p * nm * nm;
  for (int nu = 0; nu < nm; ++nu) {
    cplx acc = {0.0, 0.0};
    for (int sa = 0; sa < nm; ++sa) {
      cplx inner = {0.0, 0.0};
      for (int m = 0; m < nw; ++m) {
        cplx row = {0.0, 0.0};
        for (int np = 0; np < nw; ++np) cfma(row, Gp[(m * nw + np) * nm + sa], U0[np * nw + n]);
        cfma_conja(inner, U1[m * nw + mp], row);
      }
      cfma(acc, inner, Z[sa * nm + nu]);
    }
    g2[((int64_t)p * nw * nw + mp * nw + n) * nm + nu] = cabs2(acc);
  }
}

}  // namespace phx
