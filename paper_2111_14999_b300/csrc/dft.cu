// Stage 2 on grid q points as a separable DFT over the R_p box (Sec. 5.5 Eq. 70 evaluated
// exactly in another order).  With q = (jx/Nx, jy/Ny, jz/Nz) the phase of Eq. 13 factorises,
// e^{2 pi i q.R} = e^{2 pi i jx rx/Nx} e^{2 pi i jy ry/Ny} e^{2 pi i jz rz/Nz} with r = R mod N,
// so for every state
//   G(q)[c] = sum_rx Ex[jx][rx] sum_ry Ey[jy][ry] sum_rz Ez[jz][rz] w_R T[R][c],
// T the stage-1 output rotated to the initial band.  k_dft_z forms T and sums over rz for every (rx, ry) pair present in the R_p set
// (Zs[jz][pair][c], in HBM); k_dft_yx_elph then, for one jz and a run of jy, sums over ry into
// shared memory, finishes the x sum for the q whose final bands can reach the delta window and
// applies U_{k+q}^dagger, Z_q and the delta weights of Eq. 29 (Sec. 4.7 Eq. 61) like the fused
// tensor-core epilogue.  FP32 on the CUDA cores.
#include <algorithm>

#include <type_traits>

#include "dft.h"
#include "tc_ptx.cuh"

namespace phx {

// Sum over rz: one block per (rx plane, state); work unit = (pair of the plane, 4 jz, column
// vector).  The plane's T rows, T[R][sa][m] = w_R sum_n X[R][m][n][sa] U_k[n][b] (the rotation to the
// initial band, Eq. 71), are formed in shared memory from the stage-1 rows, read in their memory
// order; the Ez table is staged beside them.
__global__ void __launch_bounds__(256) k_dft_z(DftZArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float2 us[16];
  const int rx = blockIdx.x, s = blockIdx.y;
  const int p0 = a.plane_pair_off[rx], p1 = a.plane_pair_off[rx + 1];
  const int e0 = a.pair_ent_off[p0], ne = a.pair_ent_off[p1] - e0;
  const int E = a.E, nw = a.nw, nm = E / nw;
  float2* Ts = reinterpret_cast<float2*>(smem);            // [ne][E]
  float2* Ezs = Ts + (size_t)ne * E;                       // [Nz][Bz]
  int* azs = reinterpret_cast<int*>(Ezs + (size_t)a.Nz * a.Bz);  // [ne]
  if (threadIdx.x < nw) {
    const cplx u = a.UF[(a.gm.k_to_fine(a.st_k[s]) * nw + threadIdx.x) * nw + a.st_b[s]];
    us[threadIdx.x] = make_float2((float)u.re, (float)u.im);
  }
  __syncthreads();
  const float2* X = reinterpret_cast<const float2*>(a.X + (int64_t)a.st_kb[s] * a.ldx);
  if (nw == 8 && nm == 6) {
    // one warp per entry: the entry's 384 values X[R][m][n][sa] read in memory order as 16-byte
    // vectors, lane L holding m = L / 4 and n = 2 (L % 4), 2 (L % 4) + 1 for every sa; the sum over n
    // by two shuffle rounds among the four lanes of an m
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = lane >> 2, n0 = 2 * (lane & 3);
    const float2 u0 = us[n0], u1 = us[n0 + 1];
#pragma unroll 2  // two entries' 16-byte loads in flight per lane
    for (int e = warp; e < ne; e += (int)(blockDim.x >> 5)) {
      const int r = a.ent_r[e0 + e];
      const float4* x4 = reinterpret_cast<const float4*>(X + (int64_t)r * 384 + lane * 12);
      float2 t[6];
#pragma unroll
      for (int i = 0; i < 3; ++i) {  // n0: values 0..5, n1: values 6..11 of the lane's 12
        const float4 va = __ldg(x4 + i), vb = __ldg(x4 + 3 + i);
        const float2 a0 = make_float2(va.x, va.y), a1 = make_float2(va.z, va.w);
        const float2 b0 = make_float2(vb.x, vb.y), b1 = make_float2(vb.z, vb.w);
        t[2 * i].x = fmaf(a0.x, u0.x, fmaf(-a0.y, u0.y, fmaf(b0.x, u1.x, -b0.y * u1.y)));
        t[2 * i].y = fmaf(a0.x, u0.y, fmaf(a0.y, u0.x, fmaf(b0.x, u1.y, b0.y * u1.x)));
        t[2 * i + 1].x = fmaf(a1.x, u0.x, fmaf(-a1.y, u0.y, fmaf(b1.x, u1.x, -b1.y * u1.y)));
        t[2 * i + 1].y = fmaf(a1.x, u0.y, fmaf(a1.y, u0.x, fmaf(b1.x, u1.y, b1.y * u1.x)));
      }
#pragma unroll
      for (int o = 1; o < 4; o <<= 1)
#pragma unroll
        for (int sa = 0; sa < 6; ++sa) {
          t[sa].x += __shfl_xor_sync(0xffffffffu, t[sa].x, o);
          t[sa].y += __shfl_xor_sync(0xffffffffu, t[sa].y, o);
        }
      const float sc = a.w[r] * a.unscale;
      const int j = lane & 3;  // lanes of an m write sa = j and j + 4
#pragma unroll
      for (int sa = 0; sa < 6; ++sa)
        if (sa == j || sa == j + 4) Ts[e * E + sa * 8 + m] = make_float2(t[sa].x * sc, t[sa].y * sc);
    }
  } else
  for (int i = threadIdx.x; i < ne * E; i += blockDim.x) {  // i = (e, m, sa), sa fastest
    const int e = i / E, rem = i % E;
    const int m = rem / nm, sa = rem % nm;
    const int r = a.ent_r[e0 + e];
    const float2* x = X + ((int64_t)r * nw + m) * nw * nm + sa;
    float re = 0.f, im = 0.f;
    for (int n = 0; n < nw; ++n) {
      const float2 v = __ldg(x + n * nm);
      const float2 u = us[n];
      re = fmaf(v.x, u.x, fmaf(-v.y, u.y, re));
      im = fmaf(v.x, u.y, fmaf(v.y, u.x, im));
    }
    const float sc = a.w[r] * a.unscale;
    Ts[e * E + sa * nw + m] = make_float2(re * sc, im * sc);
  }
  for (int i = threadIdx.x; i < a.Nz * a.Bz; i += blockDim.x) Ezs[i] = a.Ez[i];
  for (int i = threadIdx.x; i < ne; i += blockDim.x) azs[i] = a.ent_az[e0 + i];
  __syncthreads();
  // jz and Nz - jz share the sums: with Ez[jz][rz] = c + i s, Z(jz) = A + B and Z(-jz) = A - B for
  // A = sum c T, B = sum i s T; units run over jz = 0 .. Nz/2 (0 and Nz/2 are their own partners,
  // s = 0 there)
  constexpr int JZ = 4;
  const int NJ = a.Nz / 2 + 1;
  const int nzq = (NJ + JZ - 1) / JZ;
  float2* Zs = a.Zs + (int64_t)s * a.Nz * a.P * E;
  if (E % 2 == 0) {
    const int EV = E / 2;
    const int units = (p1 - p0) * nzq * EV;
    for (int u = threadIdx.x; u < units; u += blockDim.x) {
      const int cv = u % EV, rest = u / EV;
      const int jq = rest % nzq, p = p0 + rest / nzq;
      float4 A[JZ], B[JZ];
#pragma unroll
      for (int i = 0; i < JZ; ++i) A[i] = B[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int e = a.pair_ent_off[p] - e0; e < a.pair_ent_off[p + 1] - e0; ++e) {
        const float4 t = reinterpret_cast<const float4*>(Ts + (size_t)e * E)[cv];
        const int az = azs[e];
#pragma unroll
        for (int i = 0; i < JZ; ++i) {
          const int jz = jq * JZ + i;
          if (jz < NJ) {
            const float2 ez = Ezs[jz * a.Bz + az];
            A[i].x = fmaf(ez.x, t.x, A[i].x);
            A[i].y = fmaf(ez.x, t.y, A[i].y);
            A[i].z = fmaf(ez.x, t.z, A[i].z);
            A[i].w = fmaf(ez.x, t.w, A[i].w);
            B[i].x = fmaf(-ez.y, t.y, B[i].x);
            B[i].y = fmaf(ez.y, t.x, B[i].y);
            B[i].z = fmaf(-ez.y, t.w, B[i].z);
            B[i].w = fmaf(ez.y, t.z, B[i].w);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < JZ; ++i) {
        const int jz = jq * JZ + i;
        if (jz < NJ) {
          reinterpret_cast<float4*>(Zs + ((int64_t)jz * a.P + p) * E)[cv] =
              make_float4(A[i].x + B[i].x, A[i].y + B[i].y, A[i].z + B[i].z, A[i].w + B[i].w);
          if (jz != 0 && 2 * jz != a.Nz)
            reinterpret_cast<float4*>(Zs + ((int64_t)(a.Nz - jz) * a.P + p) * E)[cv] =
                make_float4(A[i].x - B[i].x, A[i].y - B[i].y, A[i].z - B[i].z, A[i].w - B[i].w);
        }
      }
    }
  } else {
    const int units = (p1 - p0) * nzq * E;
    for (int u = threadIdx.x; u < units; u += blockDim.x) {
      const int cv = u % E, rest = u / E;
      const int jq = rest % nzq, p = p0 + rest / nzq;
      float2 A[JZ], B[JZ];
#pragma unroll
      for (int i = 0; i < JZ; ++i) A[i] = B[i] = make_float2(0.f, 0.f);
      for (int e = a.pair_ent_off[p] - e0; e < a.pair_ent_off[p + 1] - e0; ++e) {
        const float2 t = Ts[(size_t)e * E + cv];
        const int az = azs[e];
#pragma unroll
        for (int i = 0; i < JZ; ++i) {
          const int jz = jq * JZ + i;
          if (jz < NJ) {
            const float2 ez = Ezs[jz * a.Bz + az];
            A[i].x = fmaf(ez.x, t.x, A[i].x);
            A[i].y = fmaf(ez.x, t.y, A[i].y);
            B[i].x = fmaf(-ez.y, t.y, B[i].x);
            B[i].y = fmaf(ez.y, t.x, B[i].y);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < JZ; ++i) {
        const int jz = jq * JZ + i;
        if (jz < NJ) {
          Zs[((int64_t)jz * a.P + p) * E + cv] = make_float2(A[i].x + B[i].x, A[i].y + B[i].y);
          if (jz != 0 && 2 * jz != a.Nz)
            Zs[((int64_t)(a.Nz - jz) * a.P + p) * E + cv] = make_float2(A[i].x - B[i].x, A[i].y - B[i].y);
        }
      }
    }
  }
}

// 16-, 8- or 4-byte asynchronous global -> shared copies (cp.async).
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// 16 bytes global -> shared, bypassing L1, marked first to leave L2: for data read once (the Zs
// slices), so that it does not push the epilogue's band and phonon tables out of L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void cp_async16_stream(void* sdst, const void* gsrc, uint64_t pol) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "l"(pol)
               : "memory");
}

// N consecutive floats / complex values of a table row with the widest aligned vector loads (rows
// start on multiples of N elements, so N % 4 == 0 floats or N % 2 == 0 complex values are 16-byte aligned).
template <int N>
__device__ __forceinline__ void load_row(const float* __restrict__ p, float (&e)[N]) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(p) + i);
      e[4 * i] = v.x;
      e[4 * i + 1] = v.y;
      e[4 * i + 2] = v.z;
      e[4 * i + 3] = v.w;
    }
  } else if constexpr (N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const float2 v = __ldg(reinterpret_cast<const float2*>(p) + i);
      e[2 * i] = v.x;
      e[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) e[i] = __ldg(p + i);
  }
}
template <int N>
__device__ __forceinline__ void load_cplx(const float2* __restrict__ p, float2 (&z)[N]) {
  if constexpr (N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(p) + i);
      z[2 * i] = make_float2(v.x, v.y);
      z[2 * i + 1] = make_float2(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) z[i] = __ldg(p + i);
  }
}

// Shared-memory layout of a Y buffer: line-major, Y[line][row][c].  A row holds EP = E rounded up
// to even complex values (16-byte accesses stay aligned).  The line stride is Bx EP padded so that,
// for even NW, it is congruent to NW modulo 16: lane groups reading the same row of two consecutive
// lines (NW consecutive complex values each) then start half a bank cycle apart.
__host__ __device__ constexpr int dft_elem_stride(int E) { return E + E % 2; }
__host__ __device__ constexpr int dft_line_stride(int Bx, int E, int NW) {
  return Bx * dft_elem_stride(E) + (NW % 2 == 0 ? ((NW - Bx * dft_elem_stride(E)) % 16 + 16) % 16 : 0);
}

// x sum of NQ q (same line l, columns jx[]) over the rows of that line: real-factor rows, residue
// pairs (cos S + i sin D), residues without a partner (e^{i t r} Y).  Lane j of the group owns
// elements c = sa*NW + j*MW + mm; each row value loaded serves all NQ q.
template <int NW, int NM, int MW, int EP, int NQ>
__device__ __forceinline__ void dft_x_line(const float2* __restrict__ Yl, const float2* __restrict__ Exs,
                                           const int* __restrict__ xS, const int* __restrict__ xD, int K, int K0,
                                           int KP, const int (&jx)[NQ], int j, float2 (&G)[NQ][NM][MW]) {
#pragma unroll
  for (int u = 0; u < NQ; ++u)
#pragma unroll
    for (int sa = 0; sa < NM; ++sa)
#pragma unroll
      for (int mm = 0; mm < MW; ++mm) G[u][sa][mm] = make_float2(0.f, 0.f);
  for (int k = 0; k < K0; ++k) {
    float c[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u) c[u] = Exs[jx[u] * K + k].x;
    const float2* ys = Yl + xS[k] * EP + j * MW;
#pragma unroll
    for (int sa = 0; sa < NM; ++sa) {
      if constexpr (MW % 2 == 0) {
#pragma unroll
        for (int mm = 0; mm < MW; mm += 2) {
          const float4 v = *reinterpret_cast<const float4*>(ys + sa * NW + mm);
#pragma unroll
          for (int u = 0; u < NQ; ++u) {
            G[u][sa][mm].x = fmaf(c[u], v.x, G[u][sa][mm].x);
            G[u][sa][mm].y = fmaf(c[u], v.y, G[u][sa][mm].y);
            G[u][sa][mm + 1].x = fmaf(c[u], v.z, G[u][sa][mm + 1].x);
            G[u][sa][mm + 1].y = fmaf(c[u], v.w, G[u][sa][mm + 1].y);
          }
        }
      } else {
#pragma unroll
        for (int mm = 0; mm < MW; ++mm) {
          const float2 v = ys[sa * NW + mm];
#pragma unroll
          for (int u = 0; u < NQ; ++u) {
            G[u][sa][mm].x = fmaf(c[u], v.x, G[u][sa][mm].x);
            G[u][sa][mm].y = fmaf(c[u], v.y, G[u][sa][mm].y);
          }
        }
      }
    }
  }
#pragma unroll 2
  for (int k = K0; k < K0 + KP; ++k) {
    float2 cs[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u) cs[u] = Exs[jx[u] * K + k];
    const float2* ys = Yl + xS[k] * EP + j * MW;
    const float2* yd = Yl + xD[k] * EP + j * MW;
#pragma unroll
    for (int sa = 0; sa < NM; ++sa) {
      if constexpr (MW % 2 == 0) {
#pragma unroll
        for (int mm = 0; mm < MW; mm += 2) {
          const float4 v = *reinterpret_cast<const float4*>(ys + sa * NW + mm);
          const float4 d = *reinterpret_cast<const float4*>(yd + sa * NW + mm);
#pragma unroll
          for (int u = 0; u < NQ; ++u) {
            G[u][sa][mm].x = fmaf(cs[u].x, v.x, fmaf(-cs[u].y, d.y, G[u][sa][mm].x));
            G[u][sa][mm].y = fmaf(cs[u].x, v.y, fmaf(cs[u].y, d.x, G[u][sa][mm].y));
            G[u][sa][mm + 1].x = fmaf(cs[u].x, v.z, fmaf(-cs[u].y, d.w, G[u][sa][mm + 1].x));
            G[u][sa][mm + 1].y = fmaf(cs[u].x, v.w, fmaf(cs[u].y, d.z, G[u][sa][mm + 1].y));
          }
        }
      } else {
#pragma unroll
        for (int mm = 0; mm < MW; ++mm) {
          const float2 v = ys[sa * NW + mm], d = yd[sa * NW + mm];
#pragma unroll
          for (int u = 0; u < NQ; ++u) {
            G[u][sa][mm].x = fmaf(cs[u].x, v.x, fmaf(-cs[u].y, d.y, G[u][sa][mm].x));
            G[u][sa][mm].y = fmaf(cs[u].x, v.y, fmaf(cs[u].y, d.x, G[u][sa][mm].y));
          }
        }
      }
    }
  }
  for (int k = K0 + KP; k < K; ++k) {
    float2 ex[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u) ex[u] = Exs[jx[u] * K + k];
    const float2* y = Yl + xS[k] * EP + j * MW;
#pragma unroll
    for (int sa = 0; sa < NM; ++sa) {
      if constexpr (MW % 2 == 0) {
#pragma unroll
        for (int mm = 0; mm < MW; mm += 2) {
          const float4 v = *reinterpret_cast<const float4*>(y + sa * NW + mm);
#pragma unroll
          for (int u = 0; u < NQ; ++u) {
            G[u][sa][mm].x = fmaf(ex[u].x, v.x, fmaf(-ex[u].y, v.y, G[u][sa][mm].x));
            G[u][sa][mm].y = fmaf(ex[u].x, v.y, fmaf(ex[u].y, v.x, G[u][sa][mm].y));
            G[u][sa][mm + 1].x = fmaf(ex[u].x, v.z, fmaf(-ex[u].y, v.w, G[u][sa][mm + 1].x));
            G[u][sa][mm + 1].y = fmaf(ex[u].x, v.w, fmaf(ex[u].y, v.z, G[u][sa][mm + 1].y));
          }
        }
      } else {
#pragma unroll
        for (int mm = 0; mm < MW; ++mm) {
          const float2 v = y[sa * NW + mm];
#pragma unroll
          for (int u = 0; u < NQ; ++u) {
            G[u][sa][mm].x = fmaf(ex[u].x, v.x, fmaf(-ex[u].y, v.y, G[u][sa][mm].x));
            G[u][sa][mm].y = fmaf(ex[u].x, v.y, fmaf(ex[u].y, v.x, G[u][sa][mm].y));
          }
        }
      }
    }
  }
}

// Complex-vector helpers of the y sum: float2 = one complex value, float4 = two.
template <class V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ float4 vzero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float4 vadd(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ float4 vsub(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
// acc += c p + i s m for e = (c, s), per complex value
__device__ __forceinline__ void vcis_acc(float2& acc, float2 e, float2 p, float2 m) {
  acc.x = fmaf(e.x, p.x, fmaf(-e.y, m.y, acc.x));
  acc.y = fmaf(e.x, p.y, fmaf(e.y, m.x, acc.y));
}
__device__ __forceinline__ void vcis_acc(float4& acc, float2 e, float4 p, float4 m) {
  acc.x = fmaf(e.x, p.x, fmaf(-e.y, m.y, acc.x));
  acc.y = fmaf(e.x, p.y, fmaf(e.y, m.x, acc.y));
  acc.z = fmaf(e.x, p.z, fmaf(-e.y, m.w, acc.z));
  acc.w = fmaf(e.x, p.w, fmaf(e.y, m.z, acc.w));
}

// Adaptive Gaussian width of a pair of states (Sec. 4.7): the energy change across one mesh
// cell along each reciprocal vector, summed in quadrature over the three, over sqrt 12.
__device__ __forceinline__ float adaptive_width(const float4 va, const float4 vb, const float* __restrict__ cB,
                                                float smin) {
  const float dx = va.x - vb.x, dy = va.y - vb.y, dz = va.z - vb.z;
  float s2 = 0.f;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const float d = fmaf(dx, cB[b], fmaf(dy, cB[3 + b], dz * cB[6 + b]));
    s2 = fmaf(d, d, s2);
  }
  return fmaxf(sqrtf(s2 * (1.f / 12.f)), smin);
}

// One block per (jz, state), kDftXThreads threads; the block walks the jy lines in runs of
// kDftLines.  Loaded once: the state's Zs[jz] slice (every (rx, ry) pair) by cp.async and the
// phase tables.  Three kinds of warp task:
//  - listing (run r, 32 QR consecutive q of the run): which final bands m' at k+q can reach the
//    delta window around eps_nk; the q with at least one are appended to the run's list (warp
//    ballots, in (line, jx) order);
//  - y (run r, 32 column vectors): Y[rx][line][c] = sum_ry Ey[jy][ry] Zs[(rx,ry)][c] into one of two
//    Y buffers, the rows of residue pairs directly as S and D;
//  - x (run r, 32 / SPLIT groups of SPLIT lanes, NQ listed q of one line each): sum over the rows
//    (dft_x_line), apply U_{k+q}^dagger (partial sums over m combined by shuffles), Z_q and the delta
//    weights of every listed m'.
// Iteration r hands out from a shared counter the x tasks of run r, the y tasks of run r+1 and the
// listing tasks of run r+2 (three lists), so that warps without x work prepare the next runs.  No
// block barrier closes an iteration: each task waits for the tasks it depends on (counted per run),
// and warps that finish early go on to the next iteration.  q whose bands all miss the window
// contribute nothing to Eq. 29 and are not evaluated.
template <int NW, int NM, int SPLIT, bool PR, int NQ, bool AD, bool PL>
__global__ void __launch_bounds__(kDftXThreads, NQ == 1 ? PHX_DFT_MINB : PHX_DFT_MINB2) k_dft_yx_elph(DftXArgs a) {
  constexpr int E = NW * NM, MW = NW / SPLIT, EP = dft_elem_stride(E);
  constexpr int L = kDftLines, UL = kDftUnitLines, NWARP = kDftXThreads / 32;
  constexpr int QR = AD ? 1 : 2;         // q per lane of a listing task (the adaptive test also reads velocities)
  constexpr int XT = (32 / SPLIT) * NQ;  // list entries per x task
  static_assert(NW % SPLIT == 0 && 32 % SPLIT == 0 && NW <= 16, "lane split must divide NW and the warp");
  static_assert(SPLIT == dft_split(NW), "lane split must match the host's shared-memory sizing");
  extern __shared__ __align__(16) unsigned char smem[];
  const int P = a.P, Bx = a.Bx, By = a.By, Nx = a.Nx, Ny = a.Ny;
  const int LS = dft_line_stride(Bx, E, NW);                 // complex values per line of a Y buffer
  const int YB = L * LS;                                     // complex values per Y buffer
  float2* Zsl = reinterpret_cast<float2*>(smem);                   // [P+1][E], row P = 0
  float2* Ys = Zsl + (size_t)(P + 1) * E + ((P + 1) * E) % 2;      // [2][L][LS]
  float2* Exs = Ys + (size_t)2 * YB;                               // [Nx][K]
  float2* Eys = Exs + (size_t)Nx * a.K;                            // [Ny][By]
  int4* gidx = reinterpret_cast<int4*>(Eys + (size_t)Ny * By + (Nx * a.K + Ny * By) % 2);  // [G]
  int* gro = reinterpret_cast<int*>(gidx + a.G);                   // [K+1]
  int* gay = gro + a.K + 1;                                        // [G]
  int* xS = gay + a.G;                                             // [K]
  int* xD = xS + a.K;                                              // [K]
  int* lists = xD + a.K;                                           // [3][lcap], run r in list r % 3
  const int lcap = dft_list_cap(L, Nx);
  const int R = (Ny + L - 1) / L;
  // per run r: list length, finished listing / y / x tasks; the task counters of the iterations
  int* rc_cnt = lists + 3 * lcap;                                  // [R]
  int* rc_ldone = rc_cnt + R;                                      // [R]
  int* rc_ydone = rc_ldone + R;                                    // [R]
  int* rc_xdone = rc_ydone + R;                                    // [R]
  int* rc_task = rc_xdone + R;                                     // [R+1]: iteration r's counter at r + 1
  __shared__ int abort_s;  // a wait ran out here or in another block: the rest is skipped
  __shared__ float en_s[2];
  __shared__ double pw_s;
  __shared__ float4 vn_s;      // adaptive smearing: hbar v of the initial state
  __shared__ float2 uk_s[NW];  // polar term: U_k[m][n] of the initial state
  __shared__ double red[NWARP];
  const int s = blockIdx.y, jz = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    abort_s = *reinterpret_cast<volatile int*>(a.err);
    const double e_n = a.epsF[a.gm.k_to_fine(a.st_k[s]) * NW + a.st_b[s]];
    en_s[0] = (float)e_n;
    en_s[1] = (float)(e_n - (double)en_s[0]);
    if (AD) vn_s = a.vel[a.gm.k_to_fine(a.st_k[s]) * NW + a.st_b[s]];
    if (PL)
      for (int m = 0; m < NW; ++m) {
        const cplx u = a.UF[(a.gm.k_to_fine(a.st_k[s]) * NW + m) * NW + a.st_b[s]];
        uk_s[m] = make_float2((float)u.re, (float)u.im);
      }
    if (PR) {  // f (1 - f) / kT of the initial state (the df/de replacement of the rate)
      const double fn = 1.0 / (exp((e_n - a.mu) * a.inv_kT) + 1.0);
      pw_s = fn * (1.0 - fn) * a.inv_kT;
    }
  }
  {  // the Zs[jz] slice of this state: P * E contiguous complex values
    const float2* zg = a.Zs + ((int64_t)s * a.Nz + jz) * P * E;
    if ((P * E) % 2 == 0) {
      const uint64_t pol = l2_evict_first_policy();
      for (int i = threadIdx.x; i < P * E / 2; i += blockDim.x) cp_async16_stream(Zsl + 2 * i, zg + 2 * i, pol);
    } else {
      for (int i = threadIdx.x; i < P * E; i += blockDim.x) cp_async8(Zsl + i, zg + i);
    }
  }
  // the tables, all in flight at once beside the slice
  for (int i = threadIdx.x; i < Nx * a.K; i += blockDim.x) cp_async8(Exs + i, a.Ex + i);
  for (int i = threadIdx.x; i < Ny * By; i += blockDim.x) cp_async8(Eys + i, a.Ey + i);
  for (int i = threadIdx.x; i < a.G; i += blockDim.x) {
    cp_async16(gidx + i, a.grp_idx + i);
    cp_async4(gay + i, a.grp_ay + i);
  }
  for (int i = threadIdx.x; i <= a.K; i += blockDim.x) cp_async4(gro + i, a.row_grp_off + i);
  for (int i = threadIdx.x; i < a.K; i += blockDim.x) {
    cp_async4(xS + i, a.xS + i);
    cp_async4(xD + i, a.xD + i);
  }
  for (int i = threadIdx.x; i < E; i += blockDim.x) Zsl[(size_t)P * E + i] = make_float2(0.f, 0.f);
  for (int i = threadIdx.x; i < 5 * R + 1; i += blockDim.x) rc_cnt[i] = 0;
  int kc[3];
  grid_coords(a.gm.k_to_fine(a.st_k[s]), a.gm.nf, kc);
  // fine-grid coordinates of k+q: k_d + j_d * s_d with k_d < nf_d and j_d * s_d < nf_d, so one
  // conditional subtraction reduces them modulo nf_d
  const int sx = a.gm.sq[0], sy = a.gm.sq[1];
  const int nfx = a.gm.nf[0], nfy = a.gm.nf[1], nfz = a.gm.nf[2];
  int fz = kc[2] + jz * a.gm.sq[2];
  fz -= fz >= nfz ? nfz : 0;
  const float inv_nx = 1.f / (float)Nx;  // qi < 2^16, Nx <= 256: (qi + 0.5) / Nx truncates exactly
  cp_async_wait_all();
  __syncthreads();  // counters, en_s, tables, the slice
  const float en_hi = en_s[0], en_lo = en_s[1];
  const double pw = PR ? pw_s : 0.0;
  const float4 vn = AD ? vn_s : make_float4(0.f, 0.f, 0.f, 0.f);
  auto list_tasks = [&](int rr) { return (min(L, Ny - rr * L) * Nx + 32 * QR - 1) / (32 * QR); };

  // listing task t of run rr: q = 32 QR t + 32 u + lane of the run (u < QR), energy rows loaded
  // before any is tested
  auto list_task = [&](int rr, int t) {
    const int jy0 = rr * L;
    const int nq_run = min(L, Ny - jy0) * Nx;
    int* list = lists + (rr % 3) * lcap;
    int* cn = rc_cnt + rr;
    const int q0 = t * 32 * QR;
    float ev[QR][NW];
    int64_t kqs[QR];
    int qis[QR];
#pragma unroll
    for (int u = 0; u < QR; ++u) {
      const int qi = q0 + u * 32 + lane;
      const int l = (int)(((float)qi + 0.5f) * inv_nx);
      const int jx = qi - l * Nx;
      qis[u] = (l << 8) | jx;  // (line, jx)
      if (qi < nq_run) {
        int fx = kc[0] + jx * sx, fy = kc[1] + (jy0 + l) * sy;
        fx -= fx >= nfx ? nfx : 0;
        fy -= fy >= nfy ? nfy : 0;
        kqs[u] = (int64_t)(fx * nfy + fy) * nfz + fz;
        load_row<NW>(a.epsf + kqs[u] * NW, ev[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < QR; ++u) {
      unsigned need = 0;
      if (q0 + u * 32 + lane < nq_run) {
#pragma unroll
        for (int mp = 0; mp < NW; ++mp) {
          float reach = a.reach;
          if constexpr (AD)
            reach = (a.omega_max + a.cut * adaptive_width(vn, __ldg(a.vel + kqs[u] * NW + mp), a.cB, a.sigma_min)) *
                    1.0001f;
          if (fabsf(en_hi - ev[u][mp]) < reach) need |= 1u << mp;
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, need != 0);
      if constexpr (NQ == 1) {
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(cn, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (need) list[base + __popc(bal & ((1u << lane) - 1))] = (int)(need << 16) | qis[u];
      } else {
        // entries are consumed in pairs: each line's run of listed q in this warp is padded to an
        // even length with an entry of the same line and no band (its x sum runs, nothing else)
        const unsigned same = __match_any_sync(0xffffffffu, qis[u] >> 8);  // lanes of my line
        const unsigned bl = bal & same;
        const int first = __ffs(same) - 1;
        const bool odd_lead = lane == first && (__popc(bl) & 1);
        const unsigned oddm = __ballot_sync(0xffffffffu, odd_lead);
        const int tot = __popc(bal) + __popc(oddm);
        int base = 0;
        if (lane == 0 && tot) base = atomicAdd(cn, tot);
        base = __shfl_sync(0xffffffffu, base, 0);
        const unsigned before = (1u << first) - 1;  // lanes of the earlier lines (lines grow with lane)
        const int seg = base + __popc(bal & before) + __popc(oddm & before);
        if (need) list[seg + __popc(bl & ((1u << lane) - 1))] = (int)(need << 16) | qis[u];
        if (odd_lead) list[seg + __popc(bl)] = qis[u] & 0xffff;
      }
    }
  };

  // y task t of run rr into Y buffer rr % 2, one unit per lane; unit = (x row, kDftUnitLines lines,
  // column vector).  With Ey[jy][r] = c + i s and Ey[jy][-r] = c - i s, a y group {r, -r} adds
  // c Z+ + i s Z- to Y_a, where Z+- = Z(a, r) +- Z(a, -r).  A residue pair row k (planes a = xS[k],
  // b = xD[k]) is formed directly as S = Y_a + Y_b and D = Y_a - Y_b:
  //   S += c (Za+ + Zb+) + i s (Za- + Zb-),   D += c (Za+ - Zb+) + i s (Za- - Zb-);
  // other rows: Y_a += c Za+ + i s Za-.  Absent combinations read the zero row.  Lines past the
  // grid edge read the last Ey row (never listed, never read).
  constexpr int CV = E % 2 == 0 ? E / 2 : E;  // column vectors per row (float4 when E is even)
  using VT = typename std::conditional<E % 2 == 0, float4, float2>::type;
  const int npu = a.KP * (L / UL) * CV;
  const int units = a.K * (L / UL) * CV;
  const int y_tasks = (units + 31) / 32;
  auto y_task = [&](int rr, int t) {
    const int u = t * 32 + lane;
    if (u >= units) return;
    VT* Yb = reinterpret_cast<VT*>(Ys + (size_t)(rr & 1) * YB);
    const VT* Zv = reinterpret_cast<const VT*>(Zsl);
    constexpr int RV = E / (int)(sizeof(VT) / sizeof(float2));  // vectors per Zs / Y row
    const bool pr = u < npu;  // pair-row units first: they cost about twice as much
    const int uu = pr ? u : u - npu;
    const int cv = uu % CV, rest = uu / CV;
    const int lh = rest % (L / UL), kk = rest / (L / UL);
    const int k = pr ? a.K0 + kk : (kk < a.K0 ? kk : kk + a.KP);
    int eo[UL];
#pragma unroll
    for (int l = 0; l < UL; ++l) eo[l] = min(rr * L + lh * UL + l, Ny - 1) * By;
    VT sv[UL], dv[UL];
#pragma unroll
    for (int l = 0; l < UL; ++l) {
      sv[l] = vzero<VT>();
      dv[l] = vzero<VT>();
    }
    const int g0 = gro[k], g1 = gro[k + 1];
    if (pr) {
      for (int g = g0; g < g1; ++g) {
        const int4 gi = gidx[g];
        const VT z1 = Zv[gi.x * RV + cv], z2 = Zv[gi.y * RV + cv];
        const VT z3 = Zv[gi.z * RV + cv], z4 = Zv[gi.w * RV + cv];
        const VT ap = vadd(z1, z2), am = vsub(z1, z2), bp = vadd(z3, z4), bm = vsub(z3, z4);
        const VT ps = vadd(ap, bp), ms = vadd(am, bm), pd = vsub(ap, bp), md = vsub(am, bm);
        const int ay = gay[g];
#pragma unroll
        for (int l = 0; l < UL; ++l) {
          const float2 ey = Eys[eo[l] + ay];
          vcis_acc(sv[l], ey, ps, ms);
          vcis_acc(dv[l], ey, pd, md);
        }
      }
      const int ra = xS[k] * EP, rb = xD[k] * EP;
      constexpr int VW = (int)(sizeof(VT) / sizeof(float2));
#pragma unroll
      for (int l = 0; l < UL; ++l) {
        const size_t lo = (size_t)(lh * UL + l) * LS;
        Yb[(lo + ra) / VW + cv] = sv[l];
        Yb[(lo + rb) / VW + cv] = dv[l];
      }
    } else {
      for (int g = g0; g < g1; ++g) {
        const int4 gi = gidx[g];
        const VT z1 = Zv[gi.x * RV + cv], z2 = Zv[gi.y * RV + cv];
        const VT ap = vadd(z1, z2), am = vsub(z1, z2);
        const int ay = gay[g];
#pragma unroll
        for (int l = 0; l < UL; ++l) vcis_acc(sv[l], Eys[eo[l] + ay], ap, am);
      }
      const int ra = xS[k] * EP;
      constexpr int VW = (int)(sizeof(VT) / sizeof(float2));
#pragma unroll
      for (int l = 0; l < UL; ++l) Yb[((size_t)(lh * UL + l) * LS + ra) / VW + cv] = sv[l];
    }
  };

  const int j = threadIdx.x % SPLIT;
  const unsigned gmask = (SPLIT == 32 ? 0xffffffffu : ((1u << SPLIT) - 1)) << (lane & ~(SPLIT - 1));
  // x task t of run r: group g of the warp takes list entries XT t + NQ g .. + NQ - 1 (one line);
  // returns the lane's share of the task's Eq. 29 sum.  Every term is non-negative, so FP32 partial
  // sums lose nothing to cancellation.
  auto x_task = [&](int r, int t, int total) -> float {
    float acc = 0.f;
    const int it = t * XT + (lane / SPLIT) * NQ;
    if (it >= total) return acc;
    const float2* Yb = Ys + (size_t)(r & 1) * YB;
    const int* list = lists + (r % 3) * lcap;
    int jxs[NQ];
    unsigned needs[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      const int w = list[it + u];
      needs[u] = (unsigned)w >> 16;
      jxs[u] = w & 0xff;
    }
    const int l = (list[it] >> 8) & 0xff;
    const int jy = r * L + l;
    float2 G[NQ][NM][MW];
    dft_x_line<NW, NM, MW, EP, NQ>(Yb + (size_t)l * LS, Exs, xS, xD, a.K, a.K0, a.KP, jxs, j, G);
    int fy = kc[1] + jy * sy;
    fy -= fy >= nfy ? nfy : 0;
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      const int jx = jxs[u];
      const int q = (jx * Ny + jy) * a.Nz + jz;
      int fx = kc[0] + jx * sx;
      fx -= fx >= nfx ? nfx : 0;
      const int64_t kq = (int64_t)(fx * nfy + fy) * nfz + fz;
      const float2* zt = a.ZT + (int64_t)q * NM * NM;
      const float2* onb = a.omnb + (int64_t)q * NM;
      for (unsigned m = needs[u]; m; m &= m - 1) {
        const int mp = __ffs(m) - 1;
        const float4 el = __ldg(a.el4 + kq * NW + mp);
        const float dm = (en_hi - el.x) + (en_lo - el.y);
        const float f = el.z;
        float inv_s = a.inv_sigma, norm = 1.f;  // adaptive: 1/sigma of the pair, inside the sum
        if constexpr (AD) {
          inv_s = 1.f / adaptive_width(vn, __ldg(a.vel + kq * NW + mp), a.cB, a.sigma_min);
          norm = inv_s;
        }
        float2 uu[MW];
        load_cplx<MW>(a.UH + (kq * NW + mp) * NW + j * MW, uu);
        float2 t[NM];
#pragma unroll
        for (int sa = 0; sa < NM; ++sa) {
          t[sa] = make_float2(0.f, 0.f);
#pragma unroll
          for (int mm = 0; mm < MW; ++mm) {
            t[sa].x = fmaf(uu[mm].x, G[u][sa][mm].x, fmaf(-uu[mm].y, G[u][sa][mm].y, t[sa].x));
            t[sa].y = fmaf(uu[mm].x, G[u][sa][mm].y, fmaf(uu[mm].y, G[u][sa][mm].x, t[sa].y));
          }
        }
        float2 ov = make_float2(0.f, 0.f);  // polar term: [U_{k+q}^dagger U_k]_{m'n}, lane's m range
        if constexpr (PL) {
#pragma unroll
          for (int mm = 0; mm < MW; ++mm) {
            const float2 w = uk_s[j * MW + mm];
            ov.x = fmaf(uu[mm].x, w.x, fmaf(-uu[mm].y, w.y, ov.x));
            ov.y = fmaf(uu[mm].x, w.y, fmaf(uu[mm].y, w.x, ov.y));
          }
        }
#pragma unroll
        for (int o = 1; o < SPLIT; o <<= 1) {
#pragma unroll
          for (int sa = 0; sa < NM; ++sa) {
            t[sa].x += __shfl_xor_sync(gmask, t[sa].x, o);
            t[sa].y += __shfl_xor_sync(gmask, t[sa].y, o);
          }
          if constexpr (PL) {
            ov.x += __shfl_xor_sync(gmask, ov.x, o);
            ov.y += __shfl_xor_sync(gmask, ov.y, o);
          }
        }
        for (int v = j; v < NM; v += SPLIT) {
          float2 z[NM];
          load_cplx<NM>(zt + v * NM, z);
          float2 g = make_float2(0.f, 0.f);
#pragma unroll
          for (int sa = 0; sa < NM; ++sa) {
            g.x = fmaf(t[sa].x, z[sa].x, fmaf(-t[sa].y, z[sa].y, g.x));
            g.y = fmaf(t[sa].x, z[sa].y, fmaf(t[sa].y, z[sa].x, g.y));
          }
          if constexpr (PL) {  // + g^L = L_{q nu} [U_{k+q}^dagger U_k]_{m'n}
            const float2 lq = __ldg(a.gL + (int64_t)q * NM + v);
            g.x = fmaf(lq.x, ov.x, fmaf(-lq.y, ov.y, g.x));
            g.y = fmaf(lq.x, ov.y, fmaf(lq.y, ov.x, g.y));
          }
          const float2 on = __ldg(onb + v);
          const float t1 = (dm - on.x) * inv_s;
          const float t2 = (dm + on.x) * inv_s;
          const float g2 = g.x * g.x + g.y * g.y;
          float wgt = 0.f;
          if (t1 * t1 < a.cut2) {
            const float e1 = __expf(-t1 * t1);
            wgt += (on.y + 1.f - f) * e1;
            if constexpr (PR)  // this state's share of P_{q nu}: |g|^2 e^{-t1^2} f(1-f)/kT (emission delta)
              atomicAdd(a.pacc + (int64_t)q * NM + v, (double)(g2 * e1) * pw);
          }
          if (t2 * t2 < a.cut2) wgt += (on.y + f) * __expf(-t2 * t2);
          acc = fmaf(g2, wgt * norm, acc);
        }
      }
    }
    return acc;
  };

  double accd = 0.0;  // this warp's x tasks (every lane holds the same value)

  // Bounded wait until *c >= target.  Every lane reads the counter and then fences, so the shared-
  // memory writes that the finished tasks made before counting themselves are visible to it.  False
  // once the block gives up: the wait ran out (raising the abort flag and the error word), or
  // another warp or block ran out first.
  auto wait_for = [&](const int* c, int target) -> bool {
    const volatile int* vc = c;
    volatile int* ab = &abort_s;
    if (*vc >= target) {
      __threadfence_block();
      return true;
    }
    const unsigned long long t0 = tc::globaltimer();
    for (unsigned i = 1;; ++i) {
      __nanosleep(32);
      if (*vc >= target) {
        __threadfence_block();
        return true;
      }
      if ((i & 63u) == 0) {
        if (*ab || *reinterpret_cast<volatile int*>(a.err)) {
          *ab = 1;
          return false;
        }
        if (tc::globaltimer() - t0 > tc::kWaitLimitNs) {
          *ab = 1;
          atomicOr(a.err, 1);
          return false;
        }
      }
    }
  };
  // a finished task counts itself once all its lanes' writes are fenced
  auto finished = [&](int* c) {
    __threadfence_block();
    __syncwarp();
    if (lane == 0) atomicAdd(c, 1);
  };
  auto x_tasks_of = [&](int r) {  // once run r's listing is finished
    return (*reinterpret_cast<volatile int*>(rc_cnt + r) + XT - 1) / XT;
  };

  // Iteration r = -1 .. R-1 hands out, from its own counter, the x tasks of run r, the y tasks of
  // run r+1 and the listing tasks of run r+2 (and, at r = -1, of run 0).  There is no block barrier
  // between iterations: a task first waits (bounded) for the tasks it reads from or overwrites,
  // counted per run:
  //  - x of run r: the y tasks of run r (its listing is waited for before the iteration's count);
  //  - y of run r+1 (Y buffer (r+1) % 2) and listing of run r+2 (list (r+2) % 3): the x tasks of run r-1.
  // Those belong to earlier iterations, whose tasks were all handed out before any warp moved on,
  // so no two warps wait on each other.
  bool ok = abort_s == 0;
  for (int r = -1; r < R && ok; ++r) {
    int total = 0;
    if (r >= 0) {
      ok = wait_for(rc_ldone + r, list_tasks(r));
      if (!ok) break;
      total = *reinterpret_cast<volatile int*>(rc_cnt + r);
    }
    const int nx = (total + XT - 1) / XT;
    const int ny = r + 1 < R ? y_tasks : 0;
    const int np = r + 2 < R ? list_tasks(r + 2) : 0;
    const int n0 = r < 0 ? list_tasks(0) : 0;
    const int ntask = nx + ny + np + n0;
    for (;;) {
      int tn = 0;
      if (lane == 0) tn = atomicAdd(rc_task + r + 1, 1);
      const int t = __shfl_sync(0xffffffffu, tn, 0);
      if (t >= ntask) break;
      if (t < nx) {
        if (!(ok = wait_for(rc_ydone + r, y_tasks))) break;
        // the task's sum in a fixed order, then FP64: which warp takes which task does not change
        // the result beyond FP64 rounding
        float part = x_task(r, t, total);
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        accd += (double)part;
        finished(rc_xdone + r);
      } else {
        if (r >= 1 && !(ok = wait_for(rc_xdone + r - 1, x_tasks_of(r - 1)))) break;
        if (t < nx + ny) {
          y_task(r + 1, t - nx);
          finished(rc_ydone + r + 1);
        } else {
          const bool run0 = t >= nx + ny + np;  // the listing of run 0 (iteration -1)
          const int rl = run0 ? 0 : r + 2;
          list_task(rl, t - nx - ny - (run0 ? np : 0));
          finished(rc_ldone + rl);
        }
      }
    }
  }
  if (lane == 0) red[warp] = accd;
  __syncthreads();
  if (threadIdx.x == 0 && !abort_s) {
    double sum = 0.0;
    for (int i = 0; i < NWARP; ++i) sum += red[i];
    if (sum != 0.0) atomicAdd(a.gamma + a.s_base + s, sum * a.scale);
    // the pair count once per block, spread over four addresses (summed by the host); the listed
    // bands are not counted here (a count per listing task cost 1.5 % of the kernel)
    unsigned long long blk_nq = 0;
    for (int r = 0; r < R; ++r) blk_nq += (unsigned)rc_cnt[r];
    atomicAdd(a.nq_evaluated + 2 * (blockIdx.x & 3), blk_nq);
  }
}

template <int NW, int NM, int SPLIT, bool PR, int NQ, bool AD, bool PL = false>
static int launch_yx_t(cudaStream_t st, const DftXArgs& a, int S) {
  const size_t smem = dft_smem_bytes(a.P, a.Bx, a.By, NW, NM, a.Nx, a.Ny, a.K, a.G);
  if (allow_dynamic_smem(k_dft_yx_elph<NW, NM, SPLIT, PR, NQ, AD, PL>) != cudaSuccess) return -1;
  dim3 grid((unsigned)a.Nz, (unsigned)S);
  k_dft_yx_elph<NW, NM, SPLIT, PR, NQ, AD, PL><<<grid, kDftXThreads, smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Two q per lane group when a warp's 32 consecutive q span at most two lines (Nx >= 32).  The
// phonon-electron rates, the adaptive width and the polar term are not combined (the host
// rejects it).
template <int NW, int NM, int SPLIT>
static int launch_yx(cudaStream_t st, const DftXArgs& a, int S) {
  const bool pair = kDftQPair && a.Nx >= 32;
  if (a.gL)
    return pair ? launch_yx_t<NW, NM, SPLIT, false, 2, false, true>(st, a, S)
                : launch_yx_t<NW, NM, SPLIT, false, 1, false, true>(st, a, S);
  if (a.vel)
    return pair ? launch_yx_t<NW, NM, SPLIT, false, 2, true>(st, a, S)
                : launch_yx_t<NW, NM, SPLIT, false, 1, true>(st, a, S);
  if (a.pacc)
    return pair ? launch_yx_t<NW, NM, SPLIT, true, 2, false>(st, a, S)
                : launch_yx_t<NW, NM, SPLIT, true, 1, false>(st, a, S);
  return pair ? launch_yx_t<NW, NM, SPLIT, false, 2, false>(st, a, S)
              : launch_yx_t<NW, NM, SPLIT, false, 1, false>(st, a, S);
}

int dft_launch(cudaStream_t st, const DftZArgs& z, const DftXArgs& x, int S, int nw, int nm, int ne_plane_max) {
  const size_t sm1 = dft_z_smem_bytes(ne_plane_max, z.E, z.Nz, z.Bz);
  if (allow_dynamic_smem(k_dft_z) != cudaSuccess) return -1;
  k_dft_z<<<dim3((unsigned)x.Bx, (unsigned)S), 256, sm1, st>>>(z);
  if (cudaGetLastError() != cudaSuccess) return -1;
  if (nw == 8 && nm == 6) return launch_yx<8, 6, dft_split(8)>(st, x, S);
  if (nw == 8 && nm == 3) return launch_yx<8, 3, dft_split(8)>(st, x, S);
  if (nw == 4 && nm == 6) return launch_yx<4, 6, dft_split(4)>(st, x, S);
  if (nw == 4 && nm == 3) return launch_yx<4, 3, dft_split(4)>(st, x, S);
  if (nw == 2 && nm == 6) return launch_yx<2, 6, dft_split(2)>(st, x, S);
  if (nw == 2 && nm == 3) return launch_yx<2, 3, dft_split(2)>(st, x, S);
  if (nw == 1 && nm == 6) return launch_yx<1, 6, dft_split(1)>(st, x, S);
  if (nw == 1 && nm == 3) return launch_yx<1, 3, dft_split(1)>(st, x, S);
  return -2;
}

size_t dft_smem_bytes(int P, int Bx, int By, int nw, int nm, int Nx, int Ny, int K, int G) {
  const size_t E = (size_t)nw * nm;
  const size_t c2 = (P + 1) * E + ((P + 1) * E) % 2 + 2 * (size_t)kDftLines * dft_line_stride(Bx, (int)E, nw) +
                    (size_t)Nx * K + (size_t)Ny * By + ((size_t)Nx * K + (size_t)Ny * By) % 2;
  const size_t runs = (size_t)(Ny + kDftLines - 1) / kDftLines;
  return sizeof(float2) * c2 + sizeof(int4) * (size_t)G +
         sizeof(int) * ((size_t)K + 1 + (size_t)G + 2 * (size_t)K + 3 * (size_t)dft_list_cap(kDftLines, Nx) + 5 * runs + 1);
}

size_t dft_z_smem_bytes(int ne_plane_max, int E, int Nz, int Bz) {
  return sizeof(float2) * ((size_t)ne_plane_max * E + (size_t)Nz * Bz) + sizeof(int) * (size_t)ne_plane_max;
}

// L_{q nu} of the polar long-range coupling (Sec. 3.2, Eq. polarlong), one thread per (q, nu):
// i pref sum_G sum_s [(q+G).Z*_s.Zq[s.][nu]] e^{-x/(4 alpha)} / x, x = (q+G).eps.(q+G), over the G box
// with q+G != 0 and x / (4 alpha) < cut; FP64 sums, FP32 result.
__global__ void k_polar_q(PolarArgs a) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.Q * a.nm) return;
  const int64_t q = t / a.nm;
  const int nu = (int)(t % a.nm);
  const int j2 = (int)(q % a.N[2]), j1 = (int)((q / a.N[2]) % a.N[1]), j0 = (int)(q / ((int64_t)a.N[2] * a.N[1]));
  const double qf[3] = {(double)j0 / a.N[0], (double)j1 / a.N[1], (double)j2 / a.N[2]};
  double re = 0.0, im = 0.0;
  for (int g0 = -a.nmax[0]; g0 <= a.nmax[0]; ++g0)
    for (int g1 = -a.nmax[1]; g1 <= a.nmax[1]; ++g1)
      for (int g2 = -a.nmax[2]; g2 <= a.nmax[2]; ++g2) {
        const double f0 = qf[0] + g0, f1 = qf[1] + g1, f2 = qf[2] + g2;
        double K[3];
        for (int c = 0; c < 3; ++c) K[c] = f0 * a.B[c] + f1 * a.B[3 + c] + f2 * a.B[6 + c];
        double x = 0.0;
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c) x += K[r] * a.eps[3 * r + c] * K[c];
        if (!(x > 1e-14) || x / (4.0 * a.alpha) >= a.cut) continue;
        const double fac = exp(-x / (4.0 * a.alpha)) / x;
        for (int s = 0; s < a.na; ++s)
          for (int b = 0; b < 3; ++b) {
            const double kz = K[0] * a.zstar[9 * s + b] + K[1] * a.zstar[9 * s + 3 + b] + K[2] * a.zstar[9 * s + 6 + b];
            const cplx z = a.Zq[(q * a.nm + 3 * s + b) * a.nm + nu];
            re += fac * kz * z.re;
            im += fac * kz * z.im;
          }
      }
  a.out[t] = make_float2((float)(-a.pref * im), (float)(a.pref * re));  // i * pref * sum
}

int polar_table(cudaStream_t st, const PolarArgs& a) {
  k_polar_q<<<(unsigned)((a.Q * a.nm + 127) / 128), 128, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Phonon-electron rates from the accumulated sums (Sec. 4.3): P_{q nu} = (2 pi / N_k) n (n + 1)
// hbar w acc_{q nu} / (sqrt(pi) sigma) for live modes (0 for dead ones), then averaged over the
// modes degenerate within degen_tol at the same q.  One thread per q.
__global__ void k_prate_finish(const double* __restrict__ acc, const double* __restrict__ omega,
                               const double* __restrict__ nB, int64_t Q, int nm, double pref, double omega_cut,
                               double degen_tol, double* __restrict__ P) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= Q) return;
  double raw[32];
  for (int v = 0; v < nm; ++v) {
    const double w = omega[q * nm + v], n = nB[q * nm + v];
    raw[v] = w >= omega_cut ? pref * n * (n + 1.0) * w * acc[q * nm + v] : 0.0;
  }
  for (int v = 0; v < nm; ++v) {
    double s = 0.0;
    int c = 0;
    for (int u = 0; u < nm; ++u)
      if (fabs(omega[q * nm + u] - omega[q * nm + v]) < degen_tol) {
        s += raw[u];
        ++c;
      }
    P[q * nm + v] = s / c;
  }
}

int prate_finish(cudaStream_t st, const double* acc, const double* omega, const double* nB, int64_t Q, int nm,
                 double pref, double omega_cut, double degen_tol, double* P) {
  if (nm > 32) return -2;
  k_prate_finish<<<(unsigned)((Q + 127) / 128), 128, 0, st>>>(acc, omega, nB, Q, nm, pref, omega_cut, degen_tol, P);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// FP32 tables of the fused kernel: per fine-grid point and band the energy (window test) and
// (eps hi, eps lo, f); per q the mode factors Z[sa][v] transposed to [v][sa] and (omega, n_B).
__global__ void k_dft_tables(const double* __restrict__ epsF, const double* __restrict__ fF, int64_t NF, int nw,
                             const cplx* __restrict__ Z, const double* __restrict__ om, const double* __restrict__ nB,
                             int64_t Nq, int nm, float* __restrict__ epsf, float4* __restrict__ el4,
                             float2* __restrict__ ZT, float2* __restrict__ omnb) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < NF * nw) {
    const double e = epsF[t];
    const float hi = (float)e;
    epsf[t] = hi;
    el4[t] = make_float4(hi, (float)(e - (double)hi), (float)fF[t], 0.f);
  }
  if (t < Nq * nm * nm) {
    const int64_t q = t / (nm * nm);
    const int r = (int)(t % (nm * nm));
    const int v = r / nm, sa = r % nm;
    const cplx z = Z[q * nm * nm + sa * nm + v];
    ZT[t] = make_float2((float)z.re, (float)z.im);
  }
  if (t < Nq * nm) omnb[t] = make_float2((float)om[t], (float)nB[t]);
}

int dft_tables(cudaStream_t st, const double* epsF, const double* fF, int64_t NF, int nw, const cplx* Z,
               const double* om, const double* nB, int64_t Nq, int nm, float* epsf, float4* el4, float2* ZT,
               float2* omnb) {
  const int64_t n = NF * nw > Nq * nm * nm ? NF * nw : Nq * nm * nm;
  k_dft_tables<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(epsF, fF, NF, nw, Z, om, nB, Nq, nm, epsf, el4, ZT, omnb);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// E[j][a] = e^{2 pi i j r_a / N} for residues r_a (exact integer argument reduction, sincospi).
__global__ void k_dft_table(const int* __restrict__ res, int B, int N, float2* __restrict__ E) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * B) return;
  const int j = t / B, a = t % B;
  const int r = (int)(((int64_t)j * res[a]) % N);
  double sv, cv;
  sincospi(2.0 * (double)r / (double)N, &sv, &cv);
  E[t] = make_float2((float)cv, (float)sv);
}

int dft_table(cudaStream_t st, const int* res, int B, int N, float2* E) {
  k_dft_table<<<(N * B + 127) / 128, 128, 0, st>>>(res, B, N, E);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace phx
