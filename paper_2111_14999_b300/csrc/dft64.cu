// Both phase sums of Eq. 13 on the grids as separable DFTs (Sec. 5.5 Eqs. 70-71 evaluated exactly in
// another order), in FP64 throughout: the FP64 counterpart of dft_s1.cu and dft.cu.  Stage 1 forms
// X_k = sum_Re w e^{2 pi i k.Re} g(Re) per kx plane of the k grid (rx, then ry, then rz sums); stage 2
// rotates X to the initial band and sums over rz (k_dft_z64), then for each (jz, state) over ry into
// shared memory and, for the q whose final bands can reach the delta window, over rx, followed by
// U_{k+q}^dagger, the mode factors Z_q of Eq. 7 and the truncated Gaussians of Eq. 61 into
// Gamma_nk of Eq. 29.  The kernels are plain: one work item per thread or per warp, no task queue.
#include "dft.h"

namespace phx {

__device__ __forceinline__ double2 d2(double x, double y) { return make_double2(x, y); }
// acc += e * v (complex)
__device__ __forceinline__ void zfma(double2& acc, double2 e, double2 v) {
  acc.x = fma(e.x, v.x, fma(-e.y, v.y, acc.x));
  acc.y = fma(e.x, v.y, fma(e.y, v.x, acc.y));
}
// acc += c p + i s m for e = (c, s)
__device__ __forceinline__ void zcis(double2& acc, double2 e, double2 p, double2 m) {
  acc.x = fma(e.x, p.x, fma(-e.y, m.y, acc.x));
  acc.y = fma(e.x, p.y, fma(e.y, m.x, acc.y));
}
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return d2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return d2(a.x - b.x, a.y - b.y); }

// ---------------------------------------------------------------- stage 1
// One block per (kx plane of the batch, kS64Cols element columns), 256 threads (8 per column).
template <int GZ>
__global__ void __launch_bounds__(256) k_s1_dft64(S64Args b) {
  constexpr int CW = kS64Cols, TPC = 256 / CW;
  const S1Args& a = b.i;
  extern __shared__ __align__(16) unsigned char smem[];
  const int Pe = a.Pe, nRe = a.nRe, G = a.Gz, By = a.By;
  double2* W1 = reinterpret_cast<double2*>(smem);       // [Pe][CW]
  double2* W2 = W1 + (size_t)Pe * CW;                   // [Bz][CW]
  double2* exw = W2 + (size_t)a.Bz * CW;                // [nRe] w Ex[kx][rx] per entry
  double2* Eyk = exw + nRe;                             // [nky][By]
  double2* Ezg = Eyk + (size_t)a.nky * By;              // [nkz][G]
  int2* zg = reinterpret_cast<int2*>(Ezg + (size_t)a.nkz * G);
  int* peo = reinterpret_cast<int*>(zg + G);            // [Pe+1]
  int* erow = peo + Pe + 1;                             // [nRe]
  int* pay = erow + nRe;                                // [Pe]
  int* rzo = pay + Pe;                                  // [Bz+1]
  const int pl = blockIdx.y, kx = a.plane_kx[pl];
  const int64_t c0 = (int64_t)blockIdx.x * CW;
  const int col = threadIdx.x % CW, t8 = threadIdx.x / CW;
  const bool live = c0 + col < a.C;
  for (int i = threadIdx.x; i < nRe; i += blockDim.x) {
    const double2 e = b.Ex[kx * a.Bx + a.ent_ax[i]];
    const double w = b.ent_w[i];
    exw[i] = d2(w * e.x, w * e.y);
    erow[i] = a.ent_row[i];
  }
  for (int i = threadIdx.x; i < a.nky * By; i += blockDim.x) Eyk[i] = b.Ey[i];
  for (int i = threadIdx.x; i < a.nkz * G; i += blockDim.x) Ezg[i] = b.Ezg[i];
  for (int i = threadIdx.x; i < G; i += blockDim.x) zg[i] = a.zgrp[i];
  for (int i = threadIdx.x; i <= Pe; i += blockDim.x) peo[i] = a.pair_ent_off[i];
  for (int i = threadIdx.x; i < Pe; i += blockDim.x) pay[i] = a.pair_ay[i];
  for (int i = threadIdx.x; i <= a.Bz; i += blockDim.x) rzo[i] = a.rz_pair_off[i];
  __syncthreads();
  // rx sum: W1[p][col] = sum over the entries of (ry, rz) pair p of w Ex g
  for (int p = t8; p < Pe; p += TPC) {
    double2 acc = d2(0.0, 0.0);
    for (int e = peo[p]; e < peo[p + 1]; ++e) {
      const double2 gv = live ? __ldg(b.g + (int64_t)erow[e] * a.C + c0 + col) : d2(0.0, 0.0);
      zfma(acc, exw[e], gv);
    }
    W1[p * CW + col] = acc;
  }
  __syncthreads();
  for (int li = a.plane_line_off[pl]; li < a.plane_line_off[pl + 1]; ++li) {
    const double2* ey = Eyk + (size_t)a.line_ky[li] * By;
    for (int r = t8; r < a.Bz; r += TPC) {  // ry sum into W2(rz)
      double2 w = d2(0.0, 0.0);
      for (int p = rzo[r]; p < rzo[r + 1]; ++p) zfma(w, ey[pay[p]], W1[p * CW + col]);
      W2[r * CW + col] = w;
    }
    __syncthreads();
    // rz sum by the groups {r, -r}: Ez(r) W2(r) + Ez(-r) W2(-r) = c P + i s M
    double2 P[GZ], M[GZ];
#pragma unroll
    for (int g = 0; g < GZ; ++g) {
      P[g] = M[g] = d2(0.0, 0.0);
      if (g < G) {
        const int2 z = zg[g];
        const double2 u = W2[z.x * CW + col], v = z.y >= 0 ? W2[z.y * CW + col] : d2(0.0, 0.0);
        P[g] = zadd(u, v);
        M[g] = zsub(u, v);
      }
    }
    for (int i = a.line_k_off[li] + t8; i < a.line_k_off[li + 1]; i += TPC) {
      const int4 kr = a.kent[i];  // (kz, X row of kz, X row of -kz or -1)
      const double2* ez = Ezg + (size_t)kr.x * G;
      double2 A = d2(0.0, 0.0), B = d2(0.0, 0.0);
#pragma unroll
      for (int g = 0; g < GZ; ++g) {
        if (g >= G) break;
        const double2 e = ez[g];
        A.x = fma(e.x, P[g].x, A.x);
        A.y = fma(e.x, P[g].y, A.y);
        B.x = fma(-e.y, M[g].y, B.x);
        B.y = fma(e.y, M[g].x, B.y);
      }
      if (live) {
        b.X[(int64_t)kr.y * a.C + c0 + col] = zadd(A, B);
        if (kr.z >= 0) b.X[(int64_t)kr.z * a.C + c0 + col] = zsub(A, B);
      }
    }
    __syncthreads();  // W2 is rewritten for the next line
  }
}

size_t s64_smem_bytes(int nRe, int Pe, int Bz, int Gz, int nky, int By, int nkz) {
  return sizeof(double2) * ((size_t)Pe * kS64Cols + (size_t)Bz * kS64Cols + nRe + (size_t)nky * By + (size_t)nkz * Gz) +
         sizeof(int2) * (size_t)Gz + sizeof(int) * ((size_t)Pe + 1 + nRe + Pe + (size_t)Bz + 1);
}

template <int GZ>
static int s64_launch_t(cudaStream_t st, const S64Args& a, int planes) {
  const S1Args& i = a.i;
  const size_t smem = s64_smem_bytes(i.nRe, i.Pe, i.Bz, i.Gz, i.nky, i.By, i.nkz);
  if (allow_dynamic_smem(k_s1_dft64<GZ>) != cudaSuccess)
    return -1;
  dim3 grid((unsigned)((i.C + kS64Cols - 1) / kS64Cols), (unsigned)planes);
  k_s1_dft64<GZ><<<grid, 256, smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int s64_launch(cudaStream_t st, const S64Args& a, int planes) {
  if (planes <= 0) return 0;
  if (a.i.Gz <= 4) return s64_launch_t<4>(st, a, planes);
  if (a.i.Gz <= 8) return s64_launch_t<8>(st, a, planes);
  if (a.i.Gz <= 16) return s64_launch_t<16>(st, a, planes);
  return -2;
}

// ---------------------------------------------------------------- stage 2: z sum
// One block per (rx plane, state).  T[R][sa][m] = w_R sum_n X[R][m][n][sa] U_k[n][b] (the rotation to
// the initial band of Eq. 71) in shared memory, then Zs[jz][pair][c] = sum_rz Ez[jz][rz] T for every
// (rx, ry) pair of the plane, jz and Nz - jz sharing the cos and sin sums.
__global__ void __launch_bounds__(256) k_dft_z64(DftZ64Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double2 us[kMaxNw];
  const int rx = blockIdx.x, s = blockIdx.y;
  const int p0 = a.plane_pair_off[rx], p1 = a.plane_pair_off[rx + 1];
  const int e0 = a.pair_ent_off[p0], ne = a.pair_ent_off[p1] - e0;
  const int E = a.E, nw = a.nw, nm = E / nw;
  double2* Ts = reinterpret_cast<double2*>(smem);                  // [ne][E]
  double2* Ezs = Ts + (size_t)ne * E;                              // [Nz][Bz]
  int* azs = reinterpret_cast<int*>(Ezs + (size_t)a.Nz * a.Bz);    // [ne]
  if (threadIdx.x < nw) {
    const cplx u = a.UF[(a.gm.k_to_fine(a.st_k[s]) * nw + threadIdx.x) * nw + a.st_b[s]];
    us[threadIdx.x] = d2(u.re, u.im);
  }
  __syncthreads();
  const double2* X = a.X + (int64_t)a.st_kb[s] * a.ldx;
  for (int i = threadIdx.x; i < ne * E; i += blockDim.x) {  // i = (e, m, sa), sa fastest
    const int e = i / E, rem = i % E;
    const int m = rem / nm, sa = rem % nm;
    const int r = a.ent_r[e0 + e];
    const double2* x = X + ((int64_t)r * nw + m) * nw * nm + sa;
    double2 t = d2(0.0, 0.0);
    for (int n = 0; n < nw; ++n) zfma(t, __ldg(x + n * nm), us[n]);
    const double w = a.w[r];
    Ts[e * E + sa * nw + m] = d2(t.x * w, t.y * w);
  }
  for (int i = threadIdx.x; i < a.Nz * a.Bz; i += blockDim.x) Ezs[i] = a.Ez[i];
  for (int i = threadIdx.x; i < ne; i += blockDim.x) azs[i] = a.ent_az[e0 + i];
  __syncthreads();
  constexpr int JZ = 2;
  const int NJ = a.Nz / 2 + 1;
  const int nzq = (NJ + JZ - 1) / JZ;
  double2* Zs = a.Zs + (int64_t)s * a.Nz * a.P * E;
  const int units = (p1 - p0) * nzq * E;
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    const int c = u % E, rest = u / E;
    const int jq = rest % nzq, p = p0 + rest / nzq;
    double2 A[JZ], B[JZ];
#pragma unroll
    for (int i = 0; i < JZ; ++i) A[i] = B[i] = d2(0.0, 0.0);
    for (int e = a.pair_ent_off[p] - e0; e < a.pair_ent_off[p + 1] - e0; ++e) {
      const double2 t = Ts[(size_t)e * E + c];
      const int az = azs[e];
#pragma unroll
      for (int i = 0; i < JZ; ++i) {
        const int jz = jq * JZ + i;
        if (jz < NJ) {
          const double2 ez = Ezs[jz * a.Bz + az];
          A[i].x = fma(ez.x, t.x, A[i].x);
          A[i].y = fma(ez.x, t.y, A[i].y);
          B[i].x = fma(-ez.y, t.y, B[i].x);
          B[i].y = fma(ez.y, t.x, B[i].y);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < JZ; ++i) {
      const int jz = jq * JZ + i;
      if (jz < NJ) {
        Zs[((int64_t)jz * a.P + p) * E + c] = zadd(A[i], B[i]);
        if (jz != 0 && 2 * jz != a.Nz) Zs[((int64_t)(a.Nz - jz) * a.P + p) * E + c] = zsub(A[i], B[i]);
      }
    }
  }
}

size_t dft64_z_smem_bytes(int ne_plane_max, int E, int Nz, int Bz) {
  return sizeof(double2) * ((size_t)ne_plane_max * E + (size_t)Nz * Bz) + sizeof(int) * (size_t)ne_plane_max;
}

// ---------------------------------------------------------------- stage 2: y sum, x sum, epilogue
// One block per (jz, state), 256 threads; the state's Zs[jz] slice and the tables in shared memory.
// Per run of kDft64Lines jy lines: (1) the y sum of every x row into Y[line][plane][c] (residue pair
// rows directly as S = Y_a + Y_b and D = Y_a - Y_b, as in the FP32 kernel) and, beside it, the list of
// the run's q whose final bands can reach the delta window; (2) one warp per listed q: the x sum
// G[c] = sum over the rows, then per listed band m' one lane per mode: t[sa] = sum_m conj(U_{k+q}[m][m'])
// G[sa][m], g = sum_sa t[sa] Z_q[sa][nu] and |g|^2 times the Gaussian weights.  Bands that cannot reach
// the window contribute nothing under the truncation of Eq. 61 and are not evaluated.
__global__ void __launch_bounds__(256) k_dft_yx64(DftX64Args a) {
  constexpr int L = kDft64Lines, NWARP = 8;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int cnt[2];
  __shared__ double en_s;
  __shared__ unsigned blk_nq, blk_nb;  // the block's evaluated (state, q) pairs and listed bands
  __shared__ double red[NWARP];
  const int P = a.P, Bx = a.Bx, By = a.By, Nx = a.Nx, Ny = a.Ny, nw = a.nw, nm = a.nm, E = nw * nm;
  double2* Zsl = reinterpret_cast<double2*>(smem);          // [P+1][E], row P = 0
  double2* Ys = Zsl + (size_t)(P + 1) * E;                  // [L][Bx][E]
  double2* Exs = Ys + (size_t)L * Bx * E;                   // [Nx][K]
  double2* Eys = Exs + (size_t)Nx * a.K;                    // [Ny][By]
  double2* Gw = Eys + (size_t)Ny * By;                      // [NWARP][E]
  int4* gidx = reinterpret_cast<int4*>(Gw + (size_t)NWARP * E);  // [G]
  int* gro = reinterpret_cast<int*>(gidx + a.G);            // [K+1]
  int* gay = gro + a.K + 1;                                 // [G]
  int* xS = gay + a.G;                                      // [K]
  int* xD = xS + a.K;                                       // [K]
  int* list = xD + a.K;                                     // [L * Nx]
  const int s = blockIdx.y, jz = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t kf = a.gm.k_to_fine(a.st_k[s]);
  if (threadIdx.x == 0) {
    cnt[0] = 0;
    cnt[1] = 0;
    blk_nq = 0;
    blk_nb = 0;
    en_s = a.epsF[kf * nw + a.st_b[s]];
  }
  const double2* zg = a.Zs + ((int64_t)s * a.Nz + jz) * P * E;
  for (int i = threadIdx.x; i < P * E; i += blockDim.x) Zsl[i] = zg[i];
  for (int i = threadIdx.x; i < E; i += blockDim.x) Zsl[(size_t)P * E + i] = d2(0.0, 0.0);
  for (int i = threadIdx.x; i < Nx * a.K; i += blockDim.x) Exs[i] = a.Ex[i];
  for (int i = threadIdx.x; i < Ny * By; i += blockDim.x) Eys[i] = a.Ey[i];
  for (int i = threadIdx.x; i < a.G; i += blockDim.x) {
    gidx[i] = a.grp_idx[i];
    gay[i] = a.grp_ay[i];
  }
  for (int i = threadIdx.x; i <= a.K; i += blockDim.x) gro[i] = a.row_grp_off[i];
  for (int i = threadIdx.x; i < a.K; i += blockDim.x) {
    xS[i] = a.xS[i];
    xD[i] = a.xD[i];
  }
  int kc[3];
  grid_coords(kf, a.gm.nf, kc);
  const int nfx = a.gm.nf[0], nfy = a.gm.nf[1], nfz = a.gm.nf[2];
  int fz = kc[2] + jz * a.gm.sq[2];
  fz -= fz >= nfz ? nfz : 0;
  __syncthreads();
  const double en = en_s;
  double acc = 0.0;  // lanes < nm: this lane's share of the Eq. 29 sum
  unsigned nbands = 0;  // listed (q, band) pairs of this thread's listing
  const int R = (Ny + L - 1) / L;
  for (int r = 0; r < R; ++r) {
    const int jy0 = r * L, nl = min(L, Ny - jy0);
    if (threadIdx.x == 0) cnt[(r + 1) & 1] = 0;  // last read in iteration r - 1
    // (1a) y sum, one thread per (x row, line, element)
    const int units = a.K * nl * E;
    for (int u = threadIdx.x; u < units; u += blockDim.x) {
      const int c = u % E, rest = u / E;
      const int l = rest % nl, k = rest / nl;
      const double2* ey = Eys + (size_t)(jy0 + l) * By;
      double2* yl = Ys + (size_t)l * Bx * E;
      if (k >= a.K0 && k < a.K0 + a.KP) {  // residue pair row: S and D
        double2 S = d2(0.0, 0.0), D = d2(0.0, 0.0);
        for (int g = gro[k]; g < gro[k + 1]; ++g) {
          const int4 gi = gidx[g];
          const double2 z1 = Zsl[gi.x * E + c], z2 = Zsl[gi.y * E + c];
          const double2 z3 = Zsl[gi.z * E + c], z4 = Zsl[gi.w * E + c];
          const double2 ap = zadd(z1, z2), am = zsub(z1, z2), bp = zadd(z3, z4), bm = zsub(z3, z4);
          const double2 e = ey[gay[g]];
          zcis(S, e, zadd(ap, bp), zadd(am, bm));
          zcis(D, e, zsub(ap, bp), zsub(am, bm));
        }
        yl[xS[k] * E + c] = S;
        yl[xD[k] * E + c] = D;
      } else {
        double2 Y = d2(0.0, 0.0);
        for (int g = gro[k]; g < gro[k + 1]; ++g) {
          const int4 gi = gidx[g];
          const double2 z1 = Zsl[gi.x * E + c], z2 = Zsl[gi.y * E + c];
          zcis(Y, ey[gay[g]], zadd(z1, z2), zsub(z1, z2));
        }
        yl[xS[k] * E + c] = Y;
      }
    }
    // (1b) the run's q whose final bands can reach the window: entry = (bands << 16) | (line << 8) | jx
    for (int qi = threadIdx.x; qi < nl * Nx; qi += blockDim.x) {
      const int l = qi / Nx, jx = qi - l * Nx;
      int fx = kc[0] + jx * a.gm.sq[0], fy = kc[1] + (jy0 + l) * a.gm.sq[1];
      fx -= fx >= nfx ? nfx : 0;
      fy -= fy >= nfy ? nfy : 0;
      const int64_t kq = ((int64_t)fx * nfy + fy) * nfz + fz;
      unsigned need = 0;
      for (int mp = 0; mp < nw; ++mp)
        if (fabs(en - a.epsF[kq * nw + mp]) < a.reach) need |= 1u << mp;
      if (need) list[atomicAdd(cnt + (r & 1), 1)] = (int)(need << 16) | (l << 8) | jx;
      nbands += __popc(need);
    }
    __syncthreads();
    const int total = cnt[r & 1];
    if (threadIdx.x == 0) blk_nq += (unsigned)total;
    // (2) one warp per listed q
    double2* G = Gw + (size_t)warp * E;
    for (int it = warp; it < total; it += NWARP) {
      const int w = list[it];
      const unsigned need = (unsigned)w >> 16;
      const int l = (w >> 8) & 0xff, jx = w & 0xff, jy = jy0 + l;
      const double2* yl = Ys + (size_t)l * Bx * E;
      const double2* ex = Exs + (size_t)jx * a.K;
      for (int c = lane; c < E; c += 32) {
        double2 g = d2(0.0, 0.0);
        for (int k = 0; k < a.K0; ++k) {  // real-factor rows: cos(t r) Y
          const double2 y = yl[xS[k] * E + c];
          g.x = fma(ex[k].x, y.x, g.x);
          g.y = fma(ex[k].x, y.y, g.y);
        }
        for (int k = a.K0; k < a.K0 + a.KP; ++k)  // residue pairs: cos S + i sin D
          zcis(g, ex[k], yl[xS[k] * E + c], yl[xD[k] * E + c]);
        for (int k = a.K0 + a.KP; k < a.K; ++k) zfma(g, ex[k], yl[xS[k] * E + c]);  // e^{i t r} Y
        G[c] = g;
      }
      __syncwarp();
      const int q = (jx * Ny + jy) * a.Nz + jz;
      int fx = kc[0] + jx * a.gm.sq[0], fy = kc[1] + jy * a.gm.sq[1];
      fx -= fx >= nfx ? nfx : 0;
      fy -= fy >= nfy ? nfy : 0;
      const int64_t kq = ((int64_t)fx * nfy + fy) * nfz + fz;
      for (unsigned mset = need; mset; mset &= mset - 1) {
        const int mp = __ffs(mset) - 1;
        double2 t = d2(0.0, 0.0);  // lane sa: sum_m conj(U[m][m']) G[sa][m]
        if (lane < nm)
          for (int m = 0; m < nw; ++m) {
            const cplx u = a.UF[(kq * nw + m) * nw + mp];
            const double2 gv = G[lane * nw + m];
            t.x = fma(u.re, gv.x, fma(u.im, gv.y, t.x));
            t.y = fma(u.re, gv.y, fma(-u.im, gv.x, t.y));
          }
        double2 g = d2(0.0, 0.0);  // lane nu: sum_sa t[sa] Z_q[sa][nu]
        for (int sa = 0; sa < nm; ++sa) {
          const double tx = __shfl_sync(0xffffffffu, t.x, sa), ty = __shfl_sync(0xffffffffu, t.y, sa);
          if (lane < nm) {
            const cplx z = a.Zq[((int64_t)q * nm + sa) * nm + lane];
            g.x = fma(tx, z.re, fma(-ty, z.im, g.x));
            g.y = fma(tx, z.im, fma(ty, z.re, g.y));
          }
        }
        if (lane < nm) {
          const double om = a.omega[(int64_t)q * nm + lane], nb = a.nB[(int64_t)q * nm + lane];
          const double ep = a.epsF[kq * nw + mp], f = a.fF[kq * nw + mp];
          const double x1 = en - om - ep, x2 = en + om - ep;
          double d = 0.0;
          if (fabs(x1) < a.xcut) d += (nb + 1.0 - f) * exp(-(x1 * a.inv_sigma) * (x1 * a.inv_sigma));
          if (fabs(x2) < a.xcut) d += (nb + f) * exp(-(x2 * a.inv_sigma) * (x2 * a.inv_sigma));
          acc = fma(g.x * g.x + g.y * g.y, d, acc);
        }
      }
      __syncwarp();  // G is rewritten by the warp's next q
    }
    __syncthreads();  // Y and the list are rewritten by the next run
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  nbands = __reduce_add_sync(0xffffffffu, nbands);
  if (lane == 0 && nbands) atomicAdd(&blk_nb, nbands);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int i = 0; i < NWARP; ++i) sum += red[i];
    if (sum != 0.0) atomicAdd(a.gamma + a.s_base + s, sum * a.scale);
    unsigned long long* ctr = a.nq_evaluated + 2 * (blockIdx.x & 3);
    atomicAdd(ctr, (unsigned long long)blk_nq);
    atomicAdd(ctr + 1, (unsigned long long)blk_nb);
  }
}

size_t dft64_smem_bytes(int P, int Bx, int By, int E, int Nx, int Ny, int K, int G) {
  return sizeof(double2) * ((size_t)(P + 1) * E + (size_t)kDft64Lines * Bx * E + (size_t)Nx * K + (size_t)Ny * By +
                            (size_t)8 * E) +
         sizeof(int4) * (size_t)G + sizeof(int) * ((size_t)K + 1 + G + 2 * (size_t)K + (size_t)kDft64Lines * Nx);
}

int dft64_launch(cudaStream_t st, const DftZ64Args& z, const DftX64Args& x, int S, int ne_plane_max) {
  const size_t sm1 = dft64_z_smem_bytes(ne_plane_max, z.E, z.Nz, z.Bz);
  if (allow_dynamic_smem(k_dft_z64) != cudaSuccess) return -1;
  k_dft_z64<<<dim3((unsigned)x.Bx, (unsigned)S), 256, sm1, st>>>(z);
  if (cudaGetLastError() != cudaSuccess) return -1;
  const size_t sm2 = dft64_smem_bytes(x.P, x.Bx, x.By, x.nw * x.nm, x.Nx, x.Ny, x.K, x.G);
  if (allow_dynamic_smem(k_dft_yx64) != cudaSuccess)
    return -1;
  k_dft_yx64<<<dim3((unsigned)x.Nz, (unsigned)S), 256, sm2, st>>>(x);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// E[j][a] = e^{2 pi i j r_a / N} in FP64 (exact integer argument reduction, sincospi).
__global__ void k_dft_table64(const int* __restrict__ res, int B, int N, double2* __restrict__ E) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * B) return;
  const int j = t / B, a = t % B;
  const int r = (int)(((int64_t)j * res[a]) % N);
  double sv, cv;
  sincospi(2.0 * (double)r / (double)N, &sv, &cv);
  E[t] = d2(cv, sv);
}

int dft_table64(cudaStream_t st, const int* res, int B, int N, double2* E) {
  k_dft_table64<<<(N * B + 127) / 128, 128, 0, st>>>(res, B, N, E);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace phx
