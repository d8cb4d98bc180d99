// Reduced-precision linewidth path on tcgen05 tensor cores (sm_103a).
//
// Both phase contractions of the coupling interpolation (Sec. 5.5, Eqs. 70-71)
// are complex GEMMs P[rows][R] * X[R][cols] with a phase matrix P.  They run
// as real GEMMs through the embedding
//     A[row][2r] = Re P,  A[row][2r+1] = Im P                 (K-major, K = 2 nR)
//     B[2c][2r] = Re X,   B[2c][2r+1] = -Im X                 (K-major, N = 2 cols)
//     B[2c+1][2r] = Im X, B[2c+1][2r+1] = Re X
// so C[row][2c] = Re (P X), C[row][2c+1] = Im (P X).  Operands are split
// x = hi + lo (BF16) or big + small (TF32) and the split-precision product is
// A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation in TMEM.
//
// k_tc_gemm is one persistent, warp-specialised kernel per SM:
//   warp 0      TMA producer (one lane): A_hi, A_lo, B_hi, B_lo K-blocks into an
//               smem ring, completion signalled on "full" mbarriers
//   warp 1      TMEM allocator + MMA issuer (one lane): tcgen05.mma into one of
//               two 128 x 256 FP32 accumulators, tcgen05.commit frees smem slots
//               and publishes finished accumulators
//   warps 2-5   epilogue (128 threads = 128 TMEM lanes = the 128 tile rows),
//               overlapping the MMAs of the next tile (double-buffered TMEM)
// Epilogues: StoreEpi (stage 1: FP32 tile -> HBM) and ElphEpi (stage 2: the
// U_{k+q}^dagger / Z_q rotations, |g|^2, Gaussian delta weights and the
// Gamma accumulation, Eqs. 7, 13, 29, 61, fused so |g|^2 never reaches HBM).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdio.h>

#include "tc.h"
#include "tc_ptx.cuh"

struct TcState {
  // stage-1 B operand derived from g(Re,Rp): split parts in one operand format
  int g_key = -1;
  void* g_part[3] = {nullptr, nullptr, nullptr};
  size_t g_bytes = 0;
  float g_scale = 1.f;
};

namespace phx {

using namespace tc;

// ------------------------------------------------------------------ kernel arguments
struct TcGemmArgs {
  int m_tiles, n_tiles, kblocks, stages;
  int kb_per_chunk; // K blocks accumulated per TMEM partial
  int b_row_step;   // B rows advanced per n tile
  int group_m;      // m tiles per scheduling group (L2 reuse)
  int ntiles;       // m_tiles * n_tiles
  int* err;         // set to 1 if any bounded wait ran out
};

// Power-of-two factor that brings max|x| just below 2^14 (keeps FP16 parts in range; exact).
__host__ __device__ inline float pow2_scale(float maxabs) {
  if (!(maxabs > 0.f)) return 1.f;
  int e;
  frexpf(maxabs, &e);
  return ldexpf(1.f, 14 - e);
}

// Epilogues receive the finished FP32 tile row of their thread in registers (acc[BN],
// column c of the tile = acc[c]) and the tile coordinates.
struct StoreEpi {
  static constexpr int BN = 128;
  struct Params {
    float* C;
    int64_t ldc;
    int M, N;  // valid rows / columns of C
  };
  static __device__ __forceinline__ void tile(const Params& p, int m, int n, int b_row_step, const float* acc,
                                              int row) {
    const int64_t grow = (int64_t)m * 128 + row;
    if (grow >= p.M) return;
    const int64_t gcol0 = (int64_t)n * b_row_step;
    float* dst = p.C + grow * p.ldc + gcol0;
    if (gcol0 + BN <= p.N) {
#pragma unroll
      for (int i = 0; i < BN; i += 4) *reinterpret_cast<float4*>(dst + i) = make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
    } else {
#pragma unroll
      for (int i = 0; i < BN; ++i)
        if (gcol0 + i < p.N) dst[i] = acc[i];
    }
  }
};

template <int NW, int NM>
struct ElphEpi {
  static constexpr int CPS = 2 * NW * NM;                        // tile columns per state
  static constexpr int SPT = (128 / CPS) > 0 ? (128 / CPS) : 1;  // states per tile
  static constexpr int BN = (SPT * CPS + 15) / 16 * 16;
  struct Params {
    int Mq;                 // valid q rows
    int S;                  // states in this batch
    const int* st_k;        // batch-local state -> k grid index
    const int* st_b;        // batch-local state -> band
    int64_t s_base;         // batch offset into gamma
    GridMap gm;
    const double* epsF;     // [NF][NW]
    const float* fF;        // [NF][NW] Fermi occupations
    const float2* UH;       // [NF][NW(m')][NW(m)] = conj(U[m][m'])
    const float2* Z;        // [Nq][NM(sa)][NM(nu)]
    const float* om;        // [Nq][NM]
    const float* nB;        // [Nq][NM]
    double reach;           // omega_max + cut*sigma: |eps_n - eps_m'| beyond it contributes 0
    float inv_sigma, cut2;  // 1/sigma, cut^2
    double scale_base;      // (2 pi / N_q) / (sqrt(pi) sigma) / s_A^2
    const unsigned* tmax;   // max |T| of the batch (float bits): B operand scale pow2_scale(tmax)
    double* gamma;
  };
  static __device__ __forceinline__ void tile(const Params& p, int m, int n, int b_row_step, const float* acc,
                                              int row) {
    const float sT = pow2_scale(__uint_as_float(__ldg(p.tmax)));
    const double scale = p.scale_base / ((double)sT * (double)sT);
    const int qrow = m * 128 + row;
    const bool valid = qrow < p.Mq;
    const int q = valid ? qrow : 0;
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
      const int s = n * SPT + j;
      if (s >= p.S) break;  // uniform across the block
      const int k = __ldg(p.st_k + s);
      const int b = __ldg(p.st_b + s);
      const double eps_n = __ldg(p.epsF + p.gm.k_to_fine(k) * NW + b);
      const int64_t kq = p.gm.kq_to_fine(k, q);
      float d[NW];
      bool need = false;
#pragma unroll
      for (int mp = 0; mp < NW; ++mp) {
        double dd = eps_n - __ldg(p.epsF + kq * NW + mp);
        d[mp] = (float)dd;
        need |= valid && fabs(dd) < p.reach;
      }
      float part = 0.f;
      if (need) {
        // gz[m][nu] = sum_sa G[m][sa] Z_q[sa][nu], G[m][sa] = acc[j*CPS + 2*(sa*NW + m) + re/im]
        float2 gz[NW][NM];
#pragma unroll
        for (int mm = 0; mm < NW; ++mm)
#pragma unroll
          for (int v = 0; v < NM; ++v) gz[mm][v] = make_float2(0.f, 0.f);
#pragma unroll
        for (int sa = 0; sa < NM; ++sa) {
          float2 z[NM];
#pragma unroll
          for (int v = 0; v < NM; ++v) z[v] = __ldg(p.Z + ((int64_t)q * NM + sa) * NM + v);
#pragma unroll
          for (int mm = 0; mm < NW; ++mm) {
            const float gr = acc[j * CPS + 2 * (sa * NW + mm)], gi = acc[j * CPS + 2 * (sa * NW + mm) + 1];
#pragma unroll
            for (int v = 0; v < NM; ++v) {
              gz[mm][v].x = fmaf(gr, z[v].x, fmaf(-gi, z[v].y, gz[mm][v].x));
              gz[mm][v].y = fmaf(gr, z[v].y, fmaf(gi, z[v].x, gz[mm][v].y));
            }
          }
        }
        float om[NM], nb[NM];
#pragma unroll
        for (int v = 0; v < NM; ++v) {
          om[v] = __ldg(p.om + (int64_t)q * NM + v);
          nb[v] = __ldg(p.nB + (int64_t)q * NM + v);
        }
        for (int mp = 0; mp < NW; ++mp) {
          if (!(fabsf(d[mp]) < (float)p.reach)) continue;
          const float f = __ldg(p.fF + kq * NW + mp);
          const float2* uh = p.UH + (kq * NW + mp) * NW;
          float2 gv[NM];
#pragma unroll
          for (int v = 0; v < NM; ++v) gv[v] = make_float2(0.f, 0.f);
#pragma unroll
          for (int mm = 0; mm < NW; ++mm) {
            const float2 u = __ldg(uh + mm);
#pragma unroll
            for (int v = 0; v < NM; ++v) {
              gv[v].x = fmaf(u.x, gz[mm][v].x, fmaf(-u.y, gz[mm][v].y, gv[v].x));
              gv[v].y = fmaf(u.x, gz[mm][v].y, fmaf(u.y, gz[mm][v].x, gv[v].y));
            }
          }
#pragma unroll
          for (int v = 0; v < NM; ++v) {
            const float t1 = (d[mp] - om[v]) * p.inv_sigma;
            const float t2 = (d[mp] + om[v]) * p.inv_sigma;
            float w = 0.f;
            if (t1 * t1 < p.cut2) w += (nb[v] + 1.f - f) * expf(-t1 * t1);
            if (t2 * t2 < p.cut2) w += (nb[v] + f) * expf(-t2 * t2);
            part = fmaf(gv[v].x * gv[v].x + gv[v].y * gv[v].y, w, part);
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if ((threadIdx.x & 31) == 0 && part != 0.f) atomicAdd(p.gamma + p.s_base + s, (double)part * scale);
    }
  }
};

// ------------------------------------------------------------------ the GEMM kernel
// Accumulation.  tcgen05 FP32 accumulation rounds toward zero, which biases long
// sums low by roughly one unit in the last place per MMA.  Each K chunk (kb_per_chunk
// K blocks) is therefore accumulated in a fresh TMEM partial, and within a chunk the
// small cross products of the split parts are issued before the dominant hi*hi
// product, so the truncating steps see small accumulators.  The epilogue warps add
// the chunk partials into FP32 registers with round-to-nearest.
constexpr int kTcThreads = 192;
constexpr uint32_t kTileABytes = 128 * 128;  // 128 rows x 128 bytes (64 BF16/FP16 or 32 TF32)
constexpr int kMaxPartials = 8;

__device__ __forceinline__ void tile_coords(const TcGemmArgs& a, int t, int& m, int& n) {
  const int per_group = a.group_m * a.n_tiles;
  const int g = t / per_group;
  const int first_m = g * a.group_m;
  const int gm = min(a.group_m, a.m_tiles - first_m);
  const int r = t - g * per_group;
  m = first_m + r % gm;
  n = r / gm;
}

// Products of split parts: index 0 is the dominant hi*hi, then the corrections.
__device__ constexpr int kProdA[6] = {0, 0, 1, 0, 2, 1};
__device__ constexpr int kProdB[6] = {0, 1, 0, 2, 0, 1};

// FMT: 0 = FP16, 1 = BF16 (tcgen05 kind::f16), 2 = TF32 (kind::tf32).  NSPLIT parts per
// operand, NPROD leading products of the parts (1, 3 or 6).
template <class Epi, int FMT, int NSPLIT, int NPROD>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
              const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB0,
              const __grid_constant__ CUtensorMap tmB1, const __grid_constant__ CUtensorMap tmB2, TcGemmArgs a,
              typename Epi::Params ep) {
  constexpr int KIND = FMT == 2 ? 1 : 0;
  constexpr int BN = Epi::BN;
  constexpr uint32_t B_BYTES = (uint32_t)BN * 128u;
  constexpr uint32_t STAGE = (uint32_t)NSPLIT * (kTileABytes + B_BYTES);
  constexpr int NPART = (512 / BN) < kMaxPartials ? (512 / BN) : kMaxPartials;  // TMEM partial buffers
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)a.stages * STAGE);
  uint64_t* empty = full + a.stages;
  uint64_t* pfull = empty + a.stages;
  uint64_t* pempty = pfull + NPART;
  uint64_t* drain = pempty + NPART;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunk = (a.kblocks + a.kb_per_chunk - 1) / a.kb_per_chunk;
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.stages; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 1);
    }
    for (int i = 0; i < NPART; ++i) {
      mbar_init(pfull + i, 1);
      mbar_init(pempty + i, 128);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&tmA0);
    prefetch_tmap(&tmB0);
    if (NSPLIT > 1) {
      prefetch_tmap(&tmA1);
      prefetch_tmap(&tmB1);
    }
    if (NSPLIT > 2) {
      prefetch_tmap(&tmA2);
      prefetch_tmap(&tmB2);
    }
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int last_parity[16];
      bool armed[16];
      for (int i = 0; i < 16; ++i) armed[i] = false;
      uint32_t it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        int m, n;
        tile_coords(a, t, m, n);
        for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
          const int s = (int)(it % (uint32_t)a.stages);
          const uint32_t ph = (it / (uint32_t)a.stages) & 1u;
          if (it >= (uint32_t)a.stages && !mbar_wait(empty + s, ph ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          uint8_t* base = smem + (size_t)s * STAGE;
          mbar_arrive_expect_tx(full + s, STAGE);
          const int kx = kb * (KIND == 0 ? 64 : 32);
          uint8_t* bbase = base + NSPLIT * kTileABytes;
          tma_load_2d(base, &tmA0, full + s, kx, m * 128);
          tma_load_2d(bbase, &tmB0, full + s, kx, n * a.b_row_step);
          if (NSPLIT > 1) {
            tma_load_2d(base + kTileABytes, &tmA1, full + s, kx, m * 128);
            tma_load_2d(bbase + B_BYTES, &tmB1, full + s, kx, n * a.b_row_step);
          }
          if (NSPLIT > 2) {
            tma_load_2d(base + 2 * kTileABytes, &tmA2, full + s, kx, m * 128);
            tma_load_2d(bbase + 2 * B_BYTES, &tmB2, full + s, kx, n * a.b_row_step);
          }
          last_parity[s] = (int)ph;
          armed[s] = true;
        }
      }
      // never leave with copies in flight: wait (bounded) for the last fill of every slot
      for (int s = 0; s < a.stages; ++s) {
        if (!armed[s]) continue;
        unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(full + s, (uint32_t)last_parity[s])) {
          if (globaltimer() - t0 > kWaitLimitNs) {
            *abort_flag = 1;
            break;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      const uint32_t idesc = idesc_m128((uint32_t)BN, (uint32_t)FMT);
      uint32_t it = 0, pc = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        for (int ch = 0; ch < nchunk && ok; ++ch, ++pc) {
          const uint32_t pb = pc % (uint32_t)NPART, pph = (pc / (uint32_t)NPART) & 1u;
          if (pc >= (uint32_t)NPART && !mbar_wait(pempty + pb, pph ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + pb * (uint32_t)BN;
          const int kb0 = ch * a.kb_per_chunk, kb1 = min(a.kblocks, kb0 + a.kb_per_chunk);
          // smem slots of this chunk: wait for all of them, corrections first, then hi*hi
          uint32_t it0 = it;
          for (int kb = kb0; kb < kb1; ++kb, ++it) {
            const int s = (int)(it % (uint32_t)a.stages);
            const uint32_t ph = (it / (uint32_t)a.stages) & 1u;
            if (!mbar_wait(full + s, ph, abort_flag)) {
              ok = false;
              break;
            }
          }
          if (!ok) break;
          tc_fence_after();
          uint32_t first = 1;
#pragma unroll
          for (int pass = 0; pass < 2; ++pass) {  // pass 0: corrections, pass 1: dominant product
            for (uint32_t i2 = it0; i2 < it; ++i2) {
              const int s = (int)(i2 % (uint32_t)a.stages);
              const uint32_t abase = smem_u32(smem + (size_t)s * STAGE);
              const uint32_t bbase = abase + NSPLIT * kTileABytes;
#pragma unroll
              for (int pr = 0; pr < NPROD; ++pr) {
                if ((pass == 0) == (pr == 0)) continue;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {  // 4 MMA K-steps of 32 bytes per 128-byte row
                  const uint32_t off = (uint32_t)kk * 32u;
                  const uint64_t da = sdesc_k128(abase + kProdA[pr] * kTileABytes + off);
                  const uint64_t db = sdesc_k128(bbase + kProdB[pr] * B_BYTES + off);
                  mma<KIND>(d_tmem, da, db, idesc, first ? 0u : 1u);
                  first = 0;
                }
              }
            }
          }
          for (uint32_t i2 = it0; i2 < it; ++i2) mma_commit(empty + (int)(i2 % (uint32_t)a.stages));
          mma_commit(pfull + pb);
        }
      }
      // drain: no MMA may be in flight when TMEM is released
      mma_commit(drain);
      unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(drain, 0)) {
        if (globaltimer() - t0 > kWaitLimitNs) {
          *abort_flag = 1;
          break;
        }
      }
    }
  } else {
    // ---------------- epilogue: warps 2..5 -> TMEM lane quarters (warp % 4)
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    uint32_t pc = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
      float acc[BN];
#pragma unroll
      for (int i = 0; i < BN; ++i) acc[i] = 0.f;
      for (int ch = 0; ch < nchunk; ++ch, ++pc) {
        const uint32_t pb = pc % (uint32_t)NPART, pph = (pc / (uint32_t)NPART) & 1u;
        int w = 1;
        if (lane == 0) w = mbar_wait(pfull + pb, pph, abort_flag) ? 1 : 0;
        w = __shfl_sync(0xffffffffu, w, 0);
        if (!w) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + pb * (uint32_t)BN;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
          float v[16];
          tmem_ld16(taddr + c0, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[c0 + i] += v[i];
        }
        tc_fence_before();
        mbar_arrive(pempty + pb);
      }
      if (!ok) break;
      int m, n;
      tile_coords(a, t, m, n);
      Epi::tile(ep, m, n, a.b_row_step, acc, row);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(a.err, 1);
}

// ------------------------------------------------------------------ operand packing
// Operand formats: FP16 and BF16 (2 bytes) and TF32 (stored as FP32).
template <int FMT>
struct Fmt;
template <>
struct Fmt<0> {
  using T = __half;
  static __device__ __forceinline__ T cvt(float x) { return __float2half_rn(x); }
  static __device__ __forceinline__ float back(T v) { return __half2float(v); }
};
template <>
struct Fmt<1> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ T cvt(float x) { return __float2bfloat16_rn(x); }
  static __device__ __forceinline__ float back(T v) { return __bfloat162float(v); }
};
template <>
struct Fmt<2> {
  using T = float;
  static __device__ __forceinline__ T cvt(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
  }
  static __device__ __forceinline__ float back(T v) { return v; }
};

struct Parts {
  void* p[3];
};

// x = part0 + part1 (+ part2) + residual, each part rounded to the operand format.
template <int FMT, int NSPLIT>
__device__ __forceinline__ void split_store(float x, const Parts& P, int64_t o) {
  using T = typename Fmt<FMT>::T;
  float r = x;
#pragma unroll
  for (int i = 0; i < NSPLIT; ++i) {
    T v = Fmt<FMT>::cvt(r);
    reinterpret_cast<T*>(P.p[i])[o] = v;
    r -= Fmt<FMT>::back(v);
  }
}

// Phase operand: A[i][2r] = s w_r cos(2 pi k_i.R_r), A[i][2r+1] = s w_r sin(...), zero for 2nR <= col < Kp.
template <int FMT, int NSPLIT>
__global__ void k_pack_phase(const int* __restrict__ pts, int64_t npts, const int* __restrict__ R,
                             const double* __restrict__ w, int nR, GridPhase gp, const cplx* __restrict__ cis, int Kp,
                             float scale, Parts P) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= npts * (Kp / 2)) return;
  int64_t i = t / (Kp / 2);
  int r = (int)(t % (Kp / 2));
  float re = 0.f, im = 0.f;
  if (r < nR) {
    int64_t idx = pts ? pts[i] : i;
    int j[3];
    grid_coords(idx, gp.n, j);
    int Rv[3] = {R[3 * r], R[3 * r + 1], R[3 * r + 2]};
    cplx ph = cis[phase_index(j, Rv, gp.mult, gp.L)];
    re = (float)(ph.re * w[r] * scale);
    im = (float)(ph.im * w[r] * scale);
  }
  int64_t o = i * Kp + 2 * r;
  split_store<FMT, NSPLIT>(re, P, o);
  split_store<FMT, NSPLIT>(im, P, o + 1);
}

// Stage-1 B operand from g[Re][c] (complex FP64, scaled by s): rows 2c, 2c+1; columns 2Re, 2Re+1.
template <int FMT, int NSPLIT>
__global__ void k_pack_g(const cplx* __restrict__ g, int nRe, int64_t C, int Kp, float scale, Parts P) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= C * (Kp / 2)) return;
  int64_t c = t % C;
  int r = (int)(t / C);
  float re = 0.f, im = 0.f;
  if (r < nRe) {
    cplx v = g[(int64_t)r * C + c];
    re = (float)(v.re * scale);
    im = (float)(v.im * scale);
  }
  int64_t o0 = (2 * c) * (int64_t)Kp + 2 * r, o1 = (2 * c + 1) * (int64_t)Kp + 2 * r;
  split_store<FMT, NSPLIT>(re, P, o0);
  split_store<FMT, NSPLIT>(-im, P, o0 + 1);
  split_store<FMT, NSPLIT>(im, P, o1);
  split_store<FMT, NSPLIT>(re, P, o1 + 1);
}

// T[s][Rp][sa][m] = sum_n X[kb(s)][(Rp,m,n,sa)] U_k[n][b(s)] from the stage-1 output (FP32,
// real-embedded, multiplied by unscale); records max |component| of the batch in *tmax.
__global__ void k_pack_t(const float* __restrict__ X, int64_t ldx, float unscale, const int* __restrict__ st_kb,
                         const int* __restrict__ st_k, const int* __restrict__ st_b, GridMap gm,
                         const cplx* __restrict__ UF, int S, int nRp, int nw, int nm, float2* __restrict__ T,
                         unsigned* __restrict__ tmax) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t per_s = (int64_t)nRp * nm * nw;
  float mx = 0.f;
  if (t < per_s * S) {
    int s = (int)(t / per_s);
    int64_t rem = t % per_s;
    int rp = (int)(rem / (nm * nw));
    int sa = (int)((rem / nw) % nm);
    int m = (int)(rem % nw);
    const float* x = X + (int64_t)st_kb[s] * ldx;
    const cplx* U = UF + gm.k_to_fine(st_k[s]) * nw * nw;
    int b = st_b[s];
    float re = 0.f, im = 0.f;
    for (int n = 0; n < nw; ++n) {
      int64_t c = (((int64_t)rp * nw + m) * nw + n) * nm + sa;
      float xr = x[2 * c], xi = x[2 * c + 1];
      float ur = (float)U[n * nw + b].re, ui = (float)U[n * nw + b].im;
      re = fmaf(xr, ur, fmaf(-xi, ui, re));
      im = fmaf(xr, ui, fmaf(xi, ur, im));
    }
    re *= unscale;
    im *= unscale;
    T[t] = make_float2(re, im);
    mx = fmaxf(fabsf(re), fabsf(im));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(tmax, __float_as_uint(mx));
}

// Stage-2 B operand from T (scaled by pow2_scale(*tmax)): rows 2*(s*nm*nw + sa*nw + m) + {0,1},
// columns 2Rp + {0,1}.
template <int FMT, int NSPLIT>
__global__ void k_split_t(const float2* __restrict__ T, int S, int nRp, int nw, int nm, int Kp,
                          const unsigned* __restrict__ tmax, Parts P) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t per_s = (int64_t)nRp * nm * nw;
  if (t >= per_s * S) return;
  const float sc = pow2_scale(__uint_as_float(*tmax));
  int s = (int)(t / per_s);
  int64_t rem = t % per_s;
  int rp = (int)(rem / (nm * nw));
  int sa = (int)((rem / nw) % nm);
  int m = (int)(rem % nw);
  float2 v = T[t];
  float re = v.x * sc, im = v.y * sc;
  int64_t col = 2 * (((int64_t)s * nm + sa) * nw + m);
  int64_t o0 = col * Kp + 2 * rp, o1 = (col + 1) * Kp + 2 * rp;
  split_store<FMT, NSPLIT>(re, P, o0);
  split_store<FMT, NSPLIT>(-im, P, o0 + 1);
  split_store<FMT, NSPLIT>(im, P, o1);
  split_store<FMT, NSPLIT>(re, P, o1 + 1);
}

// FP32 epilogue tables: conj-transposed U, Fermi factors, mode factors, omega, Bose factors.
__global__ void k_tables_el(const cplx* __restrict__ UF, const double* __restrict__ fF, int64_t NF, int nw,
                            float2* __restrict__ UH, float* __restrict__ f32) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= NF * nw * nw) return;
  int64_t f = t / (nw * nw);
  int mp = (int)((t / nw) % nw), m = (int)(t % nw);
  cplx u = UF[(f * nw + m) * nw + mp];
  UH[t] = make_float2((float)u.re, (float)-u.im);
  if (m == 0) f32[f * nw + mp] = (float)fF[f * nw + mp];
}

__global__ void k_tables_ph(const cplx* __restrict__ Z, const double* __restrict__ om, const double* __restrict__ nB,
                            int64_t Q, int nm, float2* __restrict__ Zf, float* __restrict__ omf, float* __restrict__ nBf) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Q * nm * nm) return;
  Zf[t] = make_float2((float)Z[t].re, (float)Z[t].im);
  if (t < Q * nm) {
    omf[t] = (float)om[t];
    nBf[t] = (float)nB[t];
  }
}


// max over |x_i| of a double array -> *out (bits of a non-negative double, atomicMax-ordered)
__global__ void k_absmax_f64(const double* __restrict__ x, int64_t n, unsigned long long* __restrict__ out) {
  __shared__ double red[256];
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(red[0]));
}

// ------------------------------------------------------------------ host side
typedef CUresult (*PFN_encodeTiled_t)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                      const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                      CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled_t encode_fn() {
  static PFN_encodeTiled_t fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_encodeTiled_t)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// 2-D K-major operand [rows][Kp] with a 128-byte inner box and 128B swizzle.
static int make_tmap(phoebe_gpu_ctx* c, CUtensorMap* tm, const void* base, int fmt, int64_t Kp, int64_t rows,
                     uint32_t box_rows) {
  PFN_encodeTiled_t enc = encode_fn();
  if (!enc) return fail(c, PHOEBE_GPU_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const int esz = fmt == 2 ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(Kp * esz)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / esz), box_rows};
  cuuint32_t es[2] = {1, 1};
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (Kp * esz) % 16 != 0)
    return fail(c, PHOEBE_GPU_ERR_ARG, "tensor map base/stride not 16-byte aligned");
  CUtensorMapDataType dt = fmt == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                    : (fmt == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
  CUresult r = enc(tm, dt, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(c, PHOEBE_GPU_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return PHOEBE_GPU_OK;
}

static int stage_bytes(int BN, int nsplit) { return nsplit * (16384 + BN * 128); }
static int pick_stages(int BN, int nsplit) {
  int st = (227 * 1024 - 1024 - 512) / stage_bytes(BN, nsplit);
  return std::max(1, std::min(st, 8));
}

template <class Epi, int FMT, int NSPLIT, int NPROD>
static int launch_gemm(phoebe_gpu_ctx* c, const CUtensorMap* A, const CUtensorMap* B, TcGemmArgs a,
                       const typename Epi::Params& ep) {
  auto kern = k_tc_gemm<Epi, FMT, NSPLIT, NPROD>;
  a.stages = pick_stages(Epi::BN, NSPLIT);
  int sm = a.stages * stage_bytes(Epi::BN, NSPLIT) + 1024 + 512;
  CK(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  int grid = std::min(a.ntiles, c->num_sms > 0 ? c->num_sms : 148);
  if (grid <= 0) return PHOEBE_GPU_OK;
  kern<<<grid, kTcThreads, sm, c->stream>>>(A[0], A[1], A[2], B[0], B[1], B[2], a, ep);
  c->launches++;
  CK(c, cudaGetLastError());
  return PHOEBE_GPU_OK;
}

void destroy_tc_state(phoebe_gpu_ctx* c) {
  if (!c->tc) return;
  for (int i = 0; i < 3; ++i)
    if (c->tc->g_part[i]) cudaFree(c->tc->g_part[i]);
  c->mem_used -= (int64_t)c->tc->g_bytes;
  delete c->tc;
  c->tc = nullptr;
}

// Allocate NSPLIT part arrays of `count` elements of `esz` bytes under one name prefix.
static int ensure_parts(phoebe_gpu_ctx* c, const char* prefix, int nsplit, size_t count, int esz, Parts* P) {
  int st;
  for (int i = 0; i < 3; ++i) P->p[i] = nullptr;
  for (int i = 0; i < nsplit; ++i) {
    char name[64];
    snprintf(name, sizeof(name), "%s_%d", prefix, i);
    P->p[i] = ensure(c, name, count * esz, &st);
    if (!P->p[i]) return st;
  }
  return PHOEBE_GPU_OK;
}

static int part_maps(phoebe_gpu_ctx* c, CUtensorMap* tm, const Parts& P, int nsplit, int fmt, int64_t Kp,
                     int64_t rows, uint32_t box_rows) {
  for (int i = 0; i < 3; ++i) TRY(make_tmap(c, tm + i, P.p[i < nsplit ? i : 0], fmt, Kp, rows, box_rows));
  return PHOEBE_GPU_OK;
}

static float host_pow2_scale(double maxabs) { return pow2_scale((float)maxabs); }

template <int NW, int NM, int FMT, int NSPLIT, int NPROD>
static int run_tc_typed(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, const GridMap& gm, int64_t ns,
                        const std::vector<int>& hk, const int* st_k, const int* st_b, const double* epsF,
                        const cplx* UF, const double* fF, const double* omega, const double* nB, const cplx* Zq,
                        double* raw) {
  const int nw = NW, nm = NM, nRe = c->nRe, nRp = c->nRp;
  const int esz = FMT == 2 ? 4 : 2;
  const int KB = 128 / esz;  // elements per 128-byte K block
  const int Kp1 = (2 * nRe + KB - 1) / KB * KB, Kp2 = (2 * nRp + KB - 1) / KB * KB;
  const int64_t C = (int64_t)nRp * nw * nw * nm;
  const int64_t NF = (int64_t)gm.nf[0] * gm.nf[1] * gm.nf[2];
  const int64_t Nq = (int64_t)gm.nq[0] * gm.nq[1] * gm.nq[2];
  int st;
  Timer tm;
  int* err = (int*)ensure(c, "tc_err", 64, &st);
  if (!err) return st;
  CK(c, cudaMemsetAsync(err, 0, 64, c->stream));
  const float sA1 = host_pow2_scale(c->we_max), sA2 = host_pow2_scale(c->wp_max);

  // stage-1 B operand from g (cached until the next set_* or a change of operand format)
  const int key = FMT * 16 + NSPLIT;
  if (!c->tc_g_valid || !c->tc || c->tc->g_key != key) {
    destroy_tc_state(c);
    c->tc = new TcState();
    unsigned long long* gmx = (unsigned long long*)ensure(c, "tc_gmax", 64, &st);
    if (!gmx) return st;
    CK(c, cudaMemsetAsync(gmx, 0, 64, c->stream));
    k_absmax_f64<<<256, 256, 0, c->stream>>>((const double*)c->bufs["g"].p, (int64_t)nRe * C * 2, gmx);
    c->launches++;
    CK(c, cudaGetLastError());
    unsigned long long bits = 0;
    CK(c, cudaMemcpyAsync(&bits, gmx, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    double gmax;
    memcpy(&gmax, &bits, sizeof(double));
    c->tc->g_scale = host_pow2_scale(gmax);
    size_t bytes = (size_t)2 * C * Kp1 * esz;
    if (c->mem_cap > 0 && c->mem_used + (int64_t)(NSPLIT * bytes) > c->mem_cap)
      return fail(c, PHOEBE_GPU_ERR_NOMEM, "stage-1 operand of %zu bytes exceeds the memory cap", NSPLIT * bytes);
    for (int i = 0; i < NSPLIT; ++i) {
      if (cudaMalloc(&c->tc->g_part[i], bytes) != cudaSuccess) {
        cudaGetLastError();
        destroy_tc_state(c);
        return fail(c, PHOEBE_GPU_ERR_NOMEM, "cannot allocate the %zu-byte stage-1 operand", NSPLIT * bytes);
      }
      c->tc->g_bytes += bytes;
      c->mem_used += (int64_t)bytes;
    }
    Parts P{{c->tc->g_part[0], c->tc->g_part[1], c->tc->g_part[2]}};
    int64_t nt = C * (Kp1 / 2);
    k_pack_g<FMT, NSPLIT><<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>((const cplx*)c->bufs["g"].p, nRe, C,
                                                                               Kp1, c->tc->g_scale, P);
    c->launches++;
    CK(c, cudaGetLastError());
    c->tc->g_key = key;
    c->tc_g_valid = true;
  }
  Parts Pg{{c->tc->g_part[0], c->tc->g_part[1], c->tc->g_part[2]}};

  // FP32 epilogue tables
  tm.begin(c);
  float2* UH = (float2*)ensure(c, "tc_UH", sizeof(float2) * NF * nw * nw, &st);
  if (!UH) return st;
  float* f32 = (float*)ensure(c, "tc_f32", sizeof(float) * NF * nw, &st);
  if (!f32) return st;
  float2* Zf = (float2*)ensure(c, "tc_Z", sizeof(float2) * Nq * nm * nm, &st);
  if (!Zf) return st;
  float* omf = (float*)ensure(c, "tc_om", sizeof(float) * Nq * nm, &st);
  if (!omf) return st;
  float* nBf = (float*)ensure(c, "tc_nB", sizeof(float) * Nq * nm, &st);
  if (!nBf) return st;
  unsigned long long* dmax = (unsigned long long*)ensure(c, "tc_max", 64, &st);
  if (!dmax) return st;
  k_tables_el<<<(unsigned)((NF * nw * nw + 255) / 256), 256, 0, c->stream>>>(UF, fF, NF, nw, UH, f32);
  k_tables_ph<<<(unsigned)((Nq * nm * nm + 255) / 256), 256, 0, c->stream>>>(Zq, omega, nB, Nq, nm, Zf, omf, nBf);
  CK(c, cudaMemsetAsync(dmax, 0, 64, c->stream));
  k_absmax_f64<<<64, 256, 0, c->stream>>>(omega, Nq * nm, dmax);
  c->launches += 3;
  CK(c, cudaGetLastError());
  unsigned long long ombits = 0;
  CK(c, cudaMemcpyAsync(&ombits, dmax, sizeof(ombits), cudaMemcpyDeviceToHost, c->stream));

  // stage-2 A operand: q phases
  GridPhase gq = make_phase(gm.nq), gk = make_phase(gm.nk);
  cplx *cis_q, *cis_k;
  TRY(cis_table(c, gq, "cis_q", &cis_q));
  TRY(cis_table(c, gk, "cis_k", &cis_k));
  Parts PAq;
  TRY(ensure_parts(c, "tc_Aq", NSPLIT, (size_t)Nq * Kp2, esz, &PAq));
  {
    int64_t nt = Nq * (Kp2 / 2);
    k_pack_phase<FMT, NSPLIT><<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(
        nullptr, Nq, (const int*)c->bufs["Rp"].p, (const double*)c->bufs["wp"].p, nRp, gq, cis_q, Kp2, sA2, PAq);
    c->launches++;
    CK(c, cudaGetLastError());
  }
  CK(c, cudaStreamSynchronize(c->stream));
  double omega_max;
  memcpy(&omega_max, &ombits, sizeof(double));
  tm.end(c, &c->stats.stage1_ms);
  CUtensorMap tAq[3];
  TRY(part_maps(c, tAq, PAq, NSPLIT, FMT, Kp2, Nq, 128));

  // stage-2 tiling: whole states per n tile
  using EE = ElphEpi<NW, NM>;
  const int cps = EE::CPS, spt = EE::SPT;
  const int BN1 = StoreEpi::BN, BN2 = EE::BN;
  const int kb_chunk = 2;
  unsigned* tmaxp = (unsigned*)ensure(c, "tc_tmax", 64, &st);
  if (!tmaxp) return st;

  // batches of whole k points, at most max_states states each
  const int max_states = p->max_batch_states > 0 ? p->max_batch_states : 4096;
  std::vector<int> kb_list, st_kb;
  int64_t i0 = 0;
  while (i0 < ns) {
    int64_t i1 = i0;
    kb_list.clear();
    st_kb.clear();
    while (i1 < ns) {
      if (kb_list.empty() || kb_list.back() != hk[i1]) {
        int64_t j = i1;  // states of this k
        while (j < ns && hk[j] == hk[i1]) ++j;
        if (!kb_list.empty() && (i1 - i0) + (j - i1) > max_states) break;
        kb_list.push_back(hk[i1]);
      }
      st_kb.push_back((int)kb_list.size() - 1);
      ++i1;
    }
    const int S = (int)(i1 - i0);
    const int nkb = (int)kb_list.size();
    void *d_kb, *d_stkb;
    TRY(upload(c, "tc_batch_k", kb_list.data(), sizeof(int) * nkb, &d_kb));
    TRY(upload(c, "tc_batch_stkb", st_kb.data(), sizeof(int) * S, &d_stkb));

    // ---- stage 1: X[kb][2C] = sum_Re phases * g   (tensor cores, StoreEpi)
    tm.begin(c);
    Parts PAk;
    TRY(ensure_parts(c, "tc_Ak", NSPLIT, (size_t)nkb * Kp1, esz, &PAk));
    float* X = (float*)ensure(c, "tc_X", sizeof(float) * nkb * 2 * C, &st);
    if (!X) return st;
    {
      int64_t nt = (int64_t)nkb * (Kp1 / 2);
      k_pack_phase<FMT, NSPLIT><<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(
          (const int*)d_kb, nkb, (const int*)c->bufs["Re"].p, (const double*)c->bufs["we"].p, nRe, gk, cis_k, Kp1,
          sA1, PAk);
      c->launches++;
      CK(c, cudaGetLastError());
    }
    CUtensorMap tAk[3], tG[3];
    TRY(part_maps(c, tAk, PAk, NSPLIT, FMT, Kp1, nkb, 128));
    TRY(part_maps(c, tG, Pg, NSPLIT, FMT, Kp1, 2 * C, BN1));
    {
      TcGemmArgs a;
      a.m_tiles = (nkb + 127) / 128;
      a.n_tiles = (int)((2 * C + BN1 - 1) / BN1);
      a.kblocks = Kp1 / KB;
      a.kb_per_chunk = kb_chunk;
      a.b_row_step = BN1;
      a.group_m = std::max(1, a.m_tiles);
      a.ntiles = a.m_tiles * a.n_tiles;
      a.err = err;
      StoreEpi::Params ep{X, 2 * C, nkb, (int)(2 * C)};
      TRY(launch_gemm<StoreEpi, FMT, NSPLIT, NPROD>(c, tAk, tG, a, ep));
    }
    // ---- U_k rotation -> T (FP32), then the scaled split stage-2 B operand
    const int64_t rows2 = (int64_t)S * cps;
    float2* Tb = (float2*)ensure(c, "tc_T", sizeof(float2) * (size_t)S * nRp * nm * nw, &st);
    if (!Tb) return st;
    Parts PB;
    TRY(ensure_parts(c, "tc_B2", NSPLIT, (size_t)rows2 * Kp2, esz, &PB));
    for (int i = 0; i < NSPLIT; ++i) CK(c, cudaMemsetAsync(PB.p[i], 0, (size_t)rows2 * Kp2 * esz, c->stream));
    CK(c, cudaMemsetAsync(tmaxp, 0, 64, c->stream));
    {
      int64_t nt = (int64_t)S * nRp * nm * nw;
      const float unscale1 = 1.0f / (sA1 * c->tc->g_scale);
      k_pack_t<<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(X, 2 * C, unscale1, (const int*)d_stkb, st_k + i0,
                                                                     st_b + i0, gm, UF, S, nRp, nw, nm, Tb, tmaxp);
      k_split_t<FMT, NSPLIT><<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(Tb, S, nRp, nw, nm, Kp2, tmaxp, PB);
      c->launches += 2;
      CK(c, cudaGetLastError());
    }
    tm.end(c, &c->stats.stage1_ms);

    // ---- stage 2 with the fused el-ph epilogue
    CUtensorMap tB[3];
    TRY(part_maps(c, tB, PB, NSPLIT, FMT, Kp2, rows2, BN2));
    tm.begin(c);
    {
      TcGemmArgs a;
      a.m_tiles = (int)((Nq + 127) / 128);
      a.n_tiles = (S + spt - 1) / spt;
      a.kblocks = Kp2 / KB;
      a.kb_per_chunk = kb_chunk;
      a.b_row_step = spt * cps;
      a.group_m = std::min(a.m_tiles, 64);
      a.ntiles = a.m_tiles * a.n_tiles;
      a.err = err;
      typename EE::Params ep;
      ep.Mq = (int)Nq;
      ep.S = S;
      ep.st_k = st_k + i0;
      ep.st_b = st_b + i0;
      ep.s_base = i0;
      ep.gm = gm;
      ep.epsF = epsF;
      ep.fF = f32;
      ep.UH = UH;
      ep.Z = Zf;
      ep.om = omf;
      ep.nB = nBf;
      ep.reach = omega_max + p->delta_cut_sigmas * p->sigma_eV;
      ep.inv_sigma = (float)(1.0 / p->sigma_eV);
      ep.cut2 = (float)(p->delta_cut_sigmas * p->delta_cut_sigmas);
      ep.scale_base = (2.0 * kPi / (double)Nq) / (kSqrtPi * p->sigma_eV) / ((double)sA2 * (double)sA2);
      ep.tmax = tmaxp;
      ep.gamma = raw;
      TRY(launch_gemm<EE, FMT, NSPLIT, NPROD>(c, tAq, tB, a, ep));
      c->stats.stage2_launches++;
    }
    tm.end(c, &c->stats.stage2_ms);
    i0 = i1;
  }
  int herr = 0;
  CK(c, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (herr) return fail(c, PHOEBE_GPU_ERR_TIMEOUT, "a tensor-core pipeline wait ran out; results discarded");
  c->stats.pairs_executed = ns * Nq;
  c->stats.stage2_flops = 8.0 * (double)Nq * nRp * (double)ns * nw * nm;
  return PHOEBE_GPU_OK;
}

template <int NW, int NM>
static int run_tc_mode(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, const GridMap& gm, int64_t ns,
                       const std::vector<int>& hk, const int* st_k, const int* st_b, const double* epsF,
                       const cplx* UF, const double* fF, const double* omega, const double* nB, const cplx* Zq,
                       double* raw) {
#define PHX_RUN(FMT_, NS_, NP_) \
  return run_tc_typed<NW, NM, FMT_, NS_, NP_>(c, p, gm, ns, hk, st_k, st_b, epsF, UF, fF, omega, nB, Zq, raw)
  switch (p->precision) {
    case PHOEBE_PREC_SPLIT_BF16: PHX_RUN(1, 3, 6);
    case PHOEBE_PREC_SPLIT_TF32: PHX_RUN(2, 2, 3);
    case PHOEBE_PREC_BF16: PHX_RUN(1, 1, 1);
    case PHOEBE_PREC_TF32: PHX_RUN(2, 1, 1);
    case PHOEBE_PREC_SPLIT_FP16: PHX_RUN(0, 2, 3);
    case PHOEBE_PREC_BF16X3: PHX_RUN(1, 2, 3);
    default: return fail(c, PHOEBE_GPU_ERR_ARG, "unknown precision %d", p->precision);
  }
#undef PHX_RUN
}

int run_tc(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, const GridMap& gm, int64_t ns,
           const std::vector<int>& hk, const int* st_k, const int* st_b, const double* epsF, const cplx* UF,
           const double* fF, const double* omega, const double* nB, const cplx* Zq, double* raw) {
  if (c->cc < 100) return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "tensor-core precisions need an sm_10x GPU");
  const int nw = c->nw, nm = 3 * c->na;
  if (nw == 8 && nm == 6) return run_tc_mode<8, 6>(c, p, gm, ns, hk, st_k, st_b, epsF, UF, fF, omega, nB, Zq, raw);
  if (nw == 2 && nm == 3) return run_tc_mode<2, 3>(c, p, gm, ns, hk, st_k, st_b, epsF, UF, fF, omega, nB, Zq, raw);
  if (nw == 1 && nm == 3) return run_tc_mode<1, 3>(c, p, gm, ns, hk, st_k, st_b, epsF, UF, fF, omega, nB, Zq, raw);
  return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED,
              "tensor-core precisions are built for (nw, 3na) in {(8,6), (2,3), (1,3)}; got (%d, %d)", nw, nm);
}

}  // namespace phx
