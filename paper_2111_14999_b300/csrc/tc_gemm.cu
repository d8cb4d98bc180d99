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
#include "sampler.h"
#include "generic.h"
#include "dft.h"
#include "tc_ptx.cuh"

struct TcState {
  // stage-1 B operand derived from g(Re,Rp): split parts in one operand format
  int g_key = -1;
  void* g_part[3] = {nullptr, nullptr, nullptr};
  size_t g_bytes = 0;
  float g_scale = 1.f;
};

#ifndef PHX_KB_PER_CHUNK
#define PHX_KB_PER_CHUNK 2  // K blocks accumulated per TMEM partial
#endif

namespace phx {

using namespace tc;

// ------------------------------------------------------------------ kernel arguments
struct TcGemmArgs {
  int m_tiles, n_tiles, kblocks, stages;
  int kb_per_chunk; // K blocks accumulated per TMEM partial
  int b_row_step;   // B rows advanced per n tile
  int group_m;      // m tiles per scheduling group (L2 reuse)
  int ntiles;       // m_tiles * n_tiles (dense order) when tile_list is NULL
  const int2* tile_list;   // optional (m, n) list; its length is read from *ntiles_dev
  const int64_t* ntiles_dev;
  int* err;         // set to 1 if any bounded wait ran out
};


// Epilogues receive the finished FP32 tile row of their thread in registers (acc[BN],
// column c of the tile = acc[c]) and the tile coordinates.
struct StoreParams {
  float* C;
  int64_t ldc;
  int M, N;  // valid rows / columns of C
};

template <int BNW_>
struct StoreEpiT {
  static constexpr int BNW = BNW_;     // columns per epilogue warpgroup
  static constexpr int BN = 2 * BNW;   // MMA N
  static constexpr uint32_t SMEM_BYTES = 0;
  struct Pre {};
  using Params = StoreParams;
  static __device__ __forceinline__ const void* smem_src(const Params&, int) { return nullptr; }
  static __device__ __forceinline__ void prefetch(const Params&, int, int, int, int, Pre&) {}
  static __device__ __forceinline__ void tile(const Params& p, int m, int n, int wg, int row, const float* acc,
                                              const Pre&, const float2*) {
    const int64_t grow = (int64_t)m * 128 + row;
    if (grow >= p.M) return;
    const int64_t gcol0 = (int64_t)n * BN + wg * BNW;
    float* dst = p.C + grow * p.ldc + gcol0;
    if (gcol0 + BNW <= p.N && (p.ldc & 3) == 0) {  // 16-byte aligned rows: vector stores
#pragma unroll
      for (int i = 0; i < BNW; i += 4) *reinterpret_cast<float4*>(dst + i) = make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
    } else {
#pragma unroll
      for (int i = 0; i < BNW; ++i)
        if (gcol0 + i < p.N) dst[i] = acc[i];
    }
  }
};
using StoreEpi = StoreEpiT<128>;     // 256-column tiles
using StoreEpi128 = StoreEpiT<64>;   // 128-column tiles

template <int NW, int NM>
struct ElphEpi {
  static constexpr int CPS = 2 * NW * NM;  // tile columns per state
  // states per epilogue warpgroup: the most whose columns fit 128 and are a multiple of 16
  static constexpr int spw_pick() {
    for (int w = 128 / CPS; w >= 1; --w)
      if ((w * CPS) % 16 == 0) return w;
    return 0;
  }
  static constexpr int SPW = spw_pick();
  static_assert(SPW >= 1, "state column count not supported by the tile layout");
  static constexpr int SPT = 2 * SPW;      // states per tile
  static constexpr int BNW = SPW * CPS;    // columns per epilogue warpgroup
  static constexpr int BN = 2 * BNW;       // MMA N
  static constexpr int ZROW = NM * NM;     // complex mode factors per q row
  static constexpr uint32_t SMEM_BYTES = 128u * ZROW * 8u;  // the tile's Z_q block
  struct Params {
    int Mq;                 // A-operand rows (q rows incl. padding)
    int S;                  // states in this batch
    const int4* sinfo;      // per batch state: (k_f x, y, z on the fine grid, band)
    const double* eps_n;    // per batch state: initial-state energy
    int64_t s_base;         // batch offset into gamma
    GridMap gm;
    const int4* qinfo;      // per A row: (q x, y, z on the fine grid (q * sq), q or -1)
    const float2* eps2;     // [NF][NW] band energies as (hi, lo) float pairs
    const float* fF;        // [NF][NW] Fermi occupations
    const float2* UH;       // [NF][NW(m')][NW(m)] = conj(U[m][m'])
    const float2* Zr;       // [A row][NM(sa)][NM(nu)] mode factors in A-row order
    const float* omr;       // [A row][NM]
    const float* nBr;       // [A row][NM]
    float reach;            // omega_max + cut*sigma: |eps_n - eps_m'| beyond it contributes 0
    float inv_sigma, cut2;  // 1/sigma, cut^2
    double scale_base;      // (2 pi / N_q) / (sqrt(pi) sigma) / s_A^2
    const unsigned* tmax;   // max |T| of the batch (float bits): B operand scale pow2_scale(tmax)
    double* gamma;
  };
  // Per-thread values loaded before the tile's reductions so their latency is hidden.
  struct Pre {
    int4 qi;
    float om[NM], nb[NM];
  };
  static __device__ __forceinline__ const void* smem_src(const Params& p, int m) { return p.Zr + (int64_t)m * 128 * ZROW; }
  static __device__ __forceinline__ void prefetch(const Params& p, int m, int n, int wg, int row, Pre& pre) {
    const int qrow = m * 128 + row;
    pre.qi = qrow < p.Mq ? __ldg(p.qinfo + qrow) : make_int4(0, 0, 0, -1);
#pragma unroll
    for (int v = 0; v < NM; ++v) {
      pre.om[v] = __ldg(p.omr + (int64_t)qrow * NM + v);
      pre.nb[v] = __ldg(p.nBr + (int64_t)qrow * NM + v);
    }
  }
  // acc[j*CPS + 2*(sa*NW + m) + {0,1}] = G_s(q)[m][sa] (Re, Im) of state j of this warpgroup's half;
  // zs = the tile's Z_q rows in shared memory.
  static __device__ __forceinline__ void tile(const Params& p, int m, int n, int wg, int row, const float* acc,
                                              const Pre& pre, const float2* zs) {
    const float sT = pow2_scale(__uint_as_float(__ldg(p.tmax)));
    const double scale = p.scale_base / ((double)sT * (double)sT);
    const bool valid = pre.qi.w >= 0;
    const float2* zrow = zs + row * ZROW;
#pragma unroll
    for (int j = 0; j < SPW; ++j) {
      const int s = n * SPT + wg * SPW + j;
      if (s >= p.S) break;  // uniform across the warpgroup
      const int4 si = __ldg(p.sinfo + s);
      const double e_n = __ldg(p.eps_n + s);
      int f0 = si.x + pre.qi.x, f1 = si.y + pre.qi.y, f2 = si.z + pre.qi.z;  // k + q on the fine grid
      f0 -= f0 >= p.gm.nf[0] ? p.gm.nf[0] : 0;
      f1 -= f1 >= p.gm.nf[1] ? p.gm.nf[1] : 0;
      f2 -= f2 >= p.gm.nf[2] ? p.gm.nf[2] : 0;
      const int kq = (f0 * p.gm.nf[1] + f1) * p.gm.nf[2] + f2;
      const float en_hi = (float)e_n, en_lo = (float)(e_n - (double)en_hi);
      unsigned need = 0;
#pragma unroll
      for (int mp = 0; mp < NW; ++mp) {
        const float2 e = __ldg(p.eps2 + (int64_t)kq * NW + mp);
        const float dm = (en_hi - e.x) + (en_lo - e.y);  // eps_n - eps_{m', k+q}
        if (valid && fabsf(dm) < p.reach) need |= 1u << mp;
      }
      const unsigned wneed = __reduce_or_sync(0xffffffffu, need);
      float part = 0.f;
#pragma unroll 1
      for (int mp = 0; mp < NW; ++mp) {
        if (!((wneed >> mp) & 1u)) continue;  // warp-uniform
        // t[sa] = sum_m conj(U_{k+q}[m][m']) G[m][sa]
        float2 u[NW];
        const float2* uh = p.UH + ((int64_t)kq * NW + mp) * NW;
#pragma unroll
        for (int mm = 0; mm < NW; ++mm) u[mm] = __ldg(uh + mm);
        float2 t[NM];
#pragma unroll
        for (int sa = 0; sa < NM; ++sa) {
          t[sa] = make_float2(0.f, 0.f);
#pragma unroll
          for (int mm = 0; mm < NW; ++mm) {
            const float gr = acc[j * CPS + 2 * (sa * NW + mm)], gi = acc[j * CPS + 2 * (sa * NW + mm) + 1];
            t[sa].x = fmaf(u[mm].x, gr, fmaf(-u[mm].y, gi, t[sa].x));
            t[sa].y = fmaf(u[mm].x, gi, fmaf(u[mm].y, gr, t[sa].y));
          }
        }
        if (!((need >> mp) & 1u)) continue;
        // g[nu] = sum_sa t[sa] Z_q[sa][nu]  (Z_q from shared memory)
        float2 g[NM];
#pragma unroll
        for (int v = 0; v < NM; ++v) g[v] = make_float2(0.f, 0.f);
#pragma unroll
        for (int sa = 0; sa < NM; ++sa) {
#pragma unroll
          for (int v = 0; v < NM; ++v) {
            const float2 z = zrow[sa * NM + v];
            g[v].x = fmaf(t[sa].x, z.x, fmaf(-t[sa].y, z.y, g[v].x));
            g[v].y = fmaf(t[sa].x, z.y, fmaf(t[sa].y, z.x, g[v].y));
          }
        }
        const float f = __ldg(p.fF + (int64_t)kq * NW + mp);
        const float2 e = __ldg(p.eps2 + (int64_t)kq * NW + mp);
        const float dm = (en_hi - e.x) + (en_lo - e.y);
#pragma unroll
        for (int v = 0; v < NM; ++v) {
          const float t1 = (dm - pre.om[v]) * p.inv_sigma;
          const float t2 = (dm + pre.om[v]) * p.inv_sigma;
          float w = 0.f;
          if (t1 * t1 < p.cut2) w += (pre.nb[v] + 1.f - f) * expf(-t1 * t1);
          if (t2 * t2 < p.cut2) w += (pre.nb[v] + f) * expf(-t2 * t2);
          part = fmaf(g[v].x * g[v].x + g[v].y * g[v].y, w, part);
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
constexpr int kEpiGroups = 2;                      // epilogue warpgroups, each owning half the columns
constexpr int kTcThreads = 64 + 128 * kEpiGroups;  // producer warp, MMA warp, epilogue warps
constexpr uint32_t kTileABytes = 128 * 128;        // 128 rows x 128 bytes (64 BF16/FP16 or 32 TF32)
constexpr int kMaxPartials = 4;                    // TMEM partial buffers

__host__ __device__ __forceinline__ void dense_tile_coords(int group_m, int m_tiles, int n_tiles, int t, int& m,
                                                           int& n) {
  const int per_group = group_m * n_tiles;
  const int g = t / per_group;
  const int first_m = g * group_m;
  const int gm = min(group_m, m_tiles - first_m);
  const int r = t - g * per_group;
  m = first_m + r % gm;
  n = r / gm;
}

__device__ __forceinline__ void tile_coords(const TcGemmArgs& a, int t, int& m, int& n) {
  if (a.tile_list) {
    const int2 v = a.tile_list[t];
    m = v.x;
    n = v.y;
    return;
  }
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
// operand, NPROD leading products of the parts (1, 3 or 6).  Every CTA loads its own A and
// B tiles; CTAs that share an A tile find it in L2.
template <class Epi, int FMT, int NSPLIT, int NPROD>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
              const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB0,
              const __grid_constant__ CUtensorMap tmB1, const __grid_constant__ CUtensorMap tmB2, TcGemmArgs a,
              typename Epi::Params ep) {
  constexpr int KIND = FMT == 2 ? 1 : 0;
  constexpr int BN = Epi::BN, BNW = Epi::BNW;
  constexpr uint32_t B_BYTES = (uint32_t)BN * 128u;
  constexpr uint32_t STAGE = (uint32_t)NSPLIT * (kTileABytes + B_BYTES);
  constexpr int NPART = (512 / BN) < kMaxPartials ? (512 / BN) : kMaxPartials;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr uint32_t ZB = (Epi::SMEM_BYTES + 1023u) & ~1023u;  // epilogue smem block
  uint8_t* zblk = smem + (size_t)a.stages * STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(zblk + ZB);
  uint64_t* empty = full + a.stages;
  uint64_t* pfull = empty + a.stages;
  uint64_t* pempty = pfull + NPART;
  uint64_t* zfull = pempty + NPART;   // epilogue block landed
  uint64_t* zempty = zfull + 1;       // every epilogue thread finished with it
  uint64_t* drain = zempty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunk = (a.kblocks + a.kb_per_chunk - 1) / a.kb_per_chunk;
  if (a.tile_list) a.ntiles = (int)*a.ntiles_dev;  // same value in every thread
  const int cid = blockIdx.x, nclu = gridDim.x;  // persistent: tiles cid, cid + nclu, ...
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.stages; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 1);  // released by the MMA commit of the slot's last K block
    }
    for (int i = 0; i < NPART; ++i) {
      mbar_init(pfull + i, 1);
      mbar_init(pempty + i, 128 * kEpiGroups);  // every epilogue thread releases its columns
    }
    mbar_init(zfull, 1);
    mbar_init(zempty, 128 * kEpiGroups);
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
      for (int t = cid; t < a.ntiles && ok; t += nclu) {
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
          const int ay = m * 128;
          tma_load_2d(base, &tmA0, full + s, kx, ay);
          if (NSPLIT > 1) tma_load_2d(base + kTileABytes, &tmA1, full + s, kx, ay);
          if (NSPLIT > 2) tma_load_2d(base + 2 * kTileABytes, &tmA2, full + s, kx, ay);
          tma_load_2d(bbase, &tmB0, full + s, kx, n * a.b_row_step);
          if (NSPLIT > 1) tma_load_2d(bbase + B_BYTES, &tmB1, full + s, kx, n * a.b_row_step);
          if (NSPLIT > 2) tma_load_2d(bbase + 2 * B_BYTES, &tmB2, full + s, kx, n * a.b_row_step);
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
      for (int t = cid; t < a.ntiles && ok; t += nclu) {
        for (int ch = 0; ch < nchunk && ok; ++ch, ++pc) {
          const uint32_t pb = pc % (uint32_t)NPART, pph = (pc / (uint32_t)NPART) & 1u;
          uint64_t* pf = pfull + pb;
          uint64_t* pe = pempty + pb;
          if (pc >= (uint32_t)NPART && !mbar_wait(pe, pph ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + pb * (uint32_t)BN;
          const int kb0 = ch * a.kb_per_chunk, kb1 = min(a.kblocks, kb0 + a.kb_per_chunk);
          // per K block: its small cross products first, then the dominant hi*hi, then release its slot
          uint32_t first = 1;  // the chunk's first MMA starts the partial from zero
          for (int kb = kb0; kb < kb1; ++kb, ++it) {
            const int s = (int)(it % (uint32_t)a.stages);
            const uint32_t ph = (it / (uint32_t)a.stages) & 1u;
            if (!mbar_wait(full + s, ph, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t abase = smem_u32(smem + (size_t)s * STAGE);
            const uint32_t bbase = abase + NSPLIT * kTileABytes;
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {  // pass 0: corrections, pass 1: dominant product
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
            mma_commit(empty + s);
          }
          if (!ok) break;
          mma_commit(pf);
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
    // ---------------- epilogue: warpgroup wg = (warp-2)/4 owns columns [wg*BNW, (wg+1)*BNW) of
    // every tile; warp w reads TMEM lanes 32*(w%4) .. 32*(w%4)+31 = tile rows of its quarter
    const int wg = (warp - 2) >> 2;
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const bool zissuer = warp == 2 && lane == 0;  // loads the per-tile epilogue block
    bool zpending = false;
    uint32_t zcount = 0;
    if (Epi::SMEM_BYTES > 0 && zissuer && cid < a.ntiles) {
      int m0, n0;
      tile_coords(a, cid, m0, n0);
      mbar_arrive_expect_tx(zfull, Epi::SMEM_BYTES);
      bulk_load(zblk, Epi::smem_src(ep, m0), Epi::SMEM_BYTES, zfull);
      zpending = true;
    }
    uint32_t pc = 0;
    bool ok = true;
    for (int t = cid; t < a.ntiles && ok; t += nclu, ++zcount) {
      int m, n;
      tile_coords(a, t, m, n);
      typename Epi::Pre pre;
      Epi::prefetch(ep, m, n, wg, row, pre);
      float acc[BNW];
#pragma unroll
      for (int i = 0; i < BNW; ++i) acc[i] = 0.f;
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
        const uint32_t taddr =
            tmem_base + ((uint32_t)(quarter * 32) << 16) + pb * (uint32_t)BN + (uint32_t)(wg * BNW);
        if constexpr (BNW % 32 == 0) {
#pragma unroll
          for (int c0 = 0; c0 < BNW; c0 += 32) {
            float v[32];
            tmem_ld32(taddr + c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) acc[c0 + i] += v[i];
          }
        } else {
#pragma unroll
          for (int c0 = 0; c0 < BNW; c0 += 16) {
            float v[16];
            tmem_ld16(taddr + c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[c0 + i] += v[i];
          }
        }
        tc_fence_before();
        mbar_arrive(pempty + pb);
      }
      if (!ok) break;
      if (Epi::SMEM_BYTES > 0) {
        int w = 1;
        if (lane == 0) w = mbar_wait(zfull, zcount & 1u, abort_flag) ? 1 : 0;
        w = __shfl_sync(0xffffffffu, w, 0);
        if (!w) {
          ok = false;
          break;
        }
        if (zissuer) zpending = false;
      }
      Epi::tile(ep, m, n, wg, row, acc, pre, reinterpret_cast<const float2*>(zblk));
      if (Epi::SMEM_BYTES > 0) {
        mbar_arrive(zempty);
        if (zissuer && t + nclu < a.ntiles) {
          // the next tile's block may replace this one once every epilogue thread is done
          if (!mbar_wait(zempty, zcount & 1u, abort_flag)) {
            ok = false;
            break;
          }
          int m1, n1;
          tile_coords(a, t + nclu, m1, n1);
          mbar_arrive_expect_tx(zfull, Epi::SMEM_BYTES);
          bulk_load(zblk, Epi::smem_src(ep, m1), Epi::SMEM_BYTES, zfull);
          zpending = true;
        }
      }
    }
    if (zpending) {  // never leave with a bulk copy in flight
      unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(zfull, zcount & 1u)) {
        if (globaltimer() - t0 > kWaitLimitNs) {
          *abort_flag = 1;
          break;
        }
      }
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
  const int64_t idx = pts ? pts[i] : i;  // < 0: padding row
  if (r < nR && idx >= 0) {
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

// ------------------------------------------------------------------ screening (exact under the delta cutoff)
// q rows of the stage-2 A operand are ordered in compact blocks of bx x by x bz q points (z fastest
// inside a block, blocks lexicographic), each padded to 128 rows.  A (block, state) pair whose
// final-state band energies cannot come within omega_max + cut*sigma of eps_n contributes nothing.
struct QBlocks {
  int b[3];   // block shape in q-grid units
  int nb[3];  // blocks per axis
  int B[3];   // matching F-grid box shape (b * sq)
  int nbox[3];
};

// lo/hi[box][band]: min / max band energy over each aligned F-grid box.
__global__ void k_box_bounds(const double* __restrict__ epsF, GridMap gm, int nw, QBlocks qb, double* __restrict__ lo,
                             double* __restrict__ hi) {
  const int64_t nbox = (int64_t)qb.nbox[0] * qb.nbox[1] * qb.nbox[2];
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nbox * nw) return;
  const int64_t box = t / nw;
  const int band = (int)(t % nw);
  int c[3];
  grid_coords(box, qb.nbox, c);
  double mn = 1e300, mx = -1e300;
  for (int x = c[0] * qb.B[0]; x < min(gm.nf[0], (c[0] + 1) * qb.B[0]); ++x)
    for (int y = c[1] * qb.B[1]; y < min(gm.nf[1], (c[1] + 1) * qb.B[1]); ++y)
      for (int z = c[2] * qb.B[2]; z < min(gm.nf[2], (c[2] + 1) * qb.B[2]); ++z) {
        int f[3] = {x, y, z};
        double e = epsF[grid_flat(f, gm.nf) * nw + band];
        mn = fmin(mn, e);
        mx = fmax(mx, e);
      }
  lo[t] = mn;
  hi[t] = mx;
}

// flag[s][blk] = 1 if some band at some k+q, q in block blk, lies within reach of eps_n(s).
__global__ void k_screen(const int* __restrict__ st_k, const int* __restrict__ st_b, int S,
                         const double* __restrict__ epsF, GridMap gm, int nw, QBlocks qb,
                         const double* __restrict__ lo, const double* __restrict__ hi, double reach,
                         unsigned char* __restrict__ flag) {
  const int nblk = qb.nb[0] * qb.nb[1] * qb.nb[2];
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)S * nblk) return;
  const int s = (int)(t / nblk), blk = (int)(t % nblk);
  int kc[3], bc[3];
  grid_coords(st_k[s], gm.nk, kc);
  grid_coords(blk, qb.nb, bc);
  int kf[3];
  for (int i = 0; i < 3; ++i) kf[i] = kc[i] * gm.sk[i];
  const double e_n = epsF[grid_flat(kf, gm.nf) * nw + st_b[s]];
  // per axis, the distinct boxes holding (k + q) of the block
  int boxes[3][8], nbx[3];
  for (int i = 0; i < 3; ++i) {
    nbx[i] = 0;
    const int q0 = bc[i] * qb.b[i], ext = min(qb.b[i], gm.nq[i] - q0);
    for (int u = 0; u < ext && u < 8; ++u) {
      const int f = (kf[i] + (q0 + u) * gm.sq[i]) % gm.nf[i];
      const int bx = f / qb.B[i];
      bool seen = false;
      for (int v = 0; v < nbx[i]; ++v) seen |= boxes[i][v] == bx;
      if (!seen) boxes[i][nbx[i]++] = bx;
    }
  }
  unsigned char need = 0;
  for (int a = 0; a < nbx[0] && !need; ++a)
    for (int b = 0; b < nbx[1] && !need; ++b)
      for (int c = 0; c < nbx[2] && !need; ++c) {
        const int64_t box = ((int64_t)boxes[0][a] * qb.nbox[1] + boxes[1][b]) * qb.nbox[2] + boxes[2][c];
        for (int m = 0; m < nw; ++m)
          if (hi[box * nw + m] >= e_n - reach && lo[box * nw + m] <= e_n + reach) {
            need = 1;
            break;
          }
      }
  flag[t] = need;
}

// Dense stage-2 tile t (grouped order) -> 1 if any of its states needs its q block.
__global__ void k_tile_flags(const unsigned char* __restrict__ flag, int S, int nblk, int spt, int group_m,
                             int m_tiles, int n_tiles, int* __restrict__ tflag) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)m_tiles * n_tiles) return;
  int m, n;
  dense_tile_coords(group_m, m_tiles, n_tiles, (int)t, m, n);
  int need = 0;
  for (int s = n * spt; s < min(S, n * spt + spt); ++s) need |= flag[(int64_t)s * nblk + m];
  tflag[t] = need;
}

// Compacted tile list and the executed (q, state) pair count.
__global__ void k_tile_write(const int* __restrict__ tflag, const int64_t* __restrict__ off, int S, int spt,
                             int group_m, int m_tiles, int n_tiles, QBlocks qb, int nq0, int nq1, int nq2,
                             int2* __restrict__ list, unsigned long long* __restrict__ pairs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)m_tiles * n_tiles || !tflag[t]) return;
  int m, n;
  dense_tile_coords(group_m, m_tiles, n_tiles, (int)t, m, n);
  list[off[t]] = make_int2(m, n);
  int bc[3];
  grid_coords(m, qb.nb, bc);
  const int nqg[3] = {nq0, nq1, nq2};
  int rows = 1;
  for (int i = 0; i < 3; ++i) rows *= min(qb.b[i], nqg[i] - bc[i] * qb.b[i]);
  const int states = min(S, n * spt + spt) - n * spt;
  atomicAdd(pairs, (unsigned long long)rows * (unsigned long long)states);
}

// FP32 epilogue tables: conj-transposed U, Fermi factors, mode factors, omega, Bose factors.
__global__ void k_tables_el(const cplx* __restrict__ UF, const double* __restrict__ fF,
                            const double* __restrict__ epsF, int64_t NF, int nw, float2* __restrict__ UH,
                            float* __restrict__ f32, float2* __restrict__ eps2) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= NF * nw * nw) return;
  int64_t f = t / (nw * nw);
  int mp = (int)((t / nw) % nw), m = (int)(t % nw);
  cplx u = UF[(f * nw + m) * nw + mp];
  UH[t] = make_float2((float)u.re, (float)-u.im);
  if (m == 0) {
    f32[f * nw + mp] = (float)fF[f * nw + mp];
    double e = epsF[f * nw + mp];
    float hi = (float)e;
    eps2[f * nw + mp] = make_float2(hi, (float)(e - (double)hi));
  }
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
// Mode factors, energies and Bose factors in stage-2 A-row order (padding rows zero).
__global__ void k_tables_ph_rows(const cplx* __restrict__ Z, const double* __restrict__ om,
                                 const double* __restrict__ nB, const int* __restrict__ q_of_row, int64_t rows,
                                 int nm, float2* __restrict__ Zr, float* __restrict__ omr, float* __restrict__ nBr) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= rows * nm * nm) return;
  const int64_t r = t / (nm * nm);
  const int e = (int)(t % (nm * nm));
  const int q = q_of_row[r];
  cplx z = q >= 0 ? Z[(int64_t)q * nm * nm + e] : cplx{0.0, 0.0};
  Zr[t] = make_float2((float)z.re, (float)z.im);
  if (e < nm) {
    omr[r * nm + e] = q >= 0 ? (float)om[(int64_t)q * nm + e] : 0.f;
    nBr[r * nm + e] = q >= 0 ? (float)nB[(int64_t)q * nm + e] : 0.f;
  }
}

// Per batch state: k on the fine grid, band, and the initial-state energy.
__global__ void k_state_info(const int* __restrict__ st_k, const int* __restrict__ st_b, int S, GridMap gm,
                             const double* __restrict__ epsF, int nw, int4* __restrict__ sinfo,
                             double* __restrict__ eps_n) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  int kc[3];
  grid_coords(st_k[s], gm.nk, kc);
  int f[3] = {kc[0] * gm.sk[0], kc[1] * gm.sk[1], kc[2] * gm.sk[2]};
  sinfo[s] = make_int4(f[0], f[1], f[2], st_b[s]);
  eps_n[s] = epsF[grid_flat(f, gm.nf) * nw + st_b[s]];
}

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
static int pick_stages(int BN, int nsplit, int extra) {
  int st = (227 * 1024 - 1024 - 512 - extra) / stage_bytes(BN, nsplit);
  return std::max(1, std::min(st, 8));
}

// Persistent launch: one CTA per SM (or fewer when there are fewer tiles).
template <class Epi, int FMT, int NSPLIT, int NPROD>
static int launch_gemm(phoebe_gpu_ctx* c, const CUtensorMap* A, const CUtensorMap* B, TcGemmArgs a,
                       const typename Epi::Params& ep) {
  auto kern = k_tc_gemm<Epi, FMT, NSPLIT, NPROD>;
  a.stages = pick_stages(Epi::BN, NSPLIT, (int)((Epi::SMEM_BYTES + 1023u) & ~1023u));
  a.kb_per_chunk = std::max(1, std::min(a.kb_per_chunk, a.stages));  // a chunk must fit in the smem ring
  a.group_m = std::min(a.group_m, a.m_tiles);
  a.ntiles = a.m_tiles * a.n_tiles;
  int sm = a.stages * stage_bytes(Epi::BN, NSPLIT) + (int)((Epi::SMEM_BYTES + 1023u) & ~1023u) + 1024 + 512;
  CK(c, allow_dynamic_smem(kern));
  int per_sm = 0;
  CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTcThreads, sm));
  if (per_sm <= 0) return fail(c, PHOEBE_GPU_ERR_CUDA, "the tensor-core GEMM (%d B smem) does not fit on an SM", sm);
  const int sms = c->num_sms > 0 ? c->num_sms : 148;
  const int grid = std::min(sms, a.ntiles);
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

// Stage-1 B operand from g (split parts in the operand format), cached on the context until
// the next set_* call or a change of operand format.
template <int FMT, int NSPLIT>
static int ensure_g_operand(phoebe_gpu_ctx* c, int64_t C, int Kp1, int esz) {
  const int nRe = c->nRe;
  int st;
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
  return PHOEBE_GPU_OK;
}

// The next batch of whole k points starting at state i0 (states ordered by k): at most
// max_states states unless a single k has more.  Returns the end state; fills the batch's k
// list and each state's index into it.
static int64_t next_batch(const std::vector<int>& hk, int64_t ns, int64_t i0, int max_states, std::vector<int>* kb_list,
                          std::vector<int>* st_kb) {
  int64_t i1 = i0;
  kb_list->clear();
  st_kb->clear();
  while (i1 < ns) {
    if (kb_list->empty() || kb_list->back() != hk[i1]) {
      int64_t j = i1;
      while (j < ns && hk[j] == hk[i1]) ++j;
      if (!kb_list->empty() && (i1 - i0) + (j - i1) > max_states) break;
      kb_list->push_back(hk[i1]);
    }
    st_kb->push_back((int)kb_list->size() - 1);
    ++i1;
  }
  return i1;
}

// Like next_batch, but the batch ends on a kx-plane boundary of the k grid when it holds more than
// one plane (the separable stage 1 then reads each plane's R_e terms once per step).
static int64_t next_batch_planes(const std::vector<int>& hk, int64_t ns, int64_t i0, int max_states, const int nk[3],
                                 std::vector<int>* kb_list, std::vector<int>* st_kb) {
  int64_t i1 = next_batch(hk, ns, i0, max_states, kb_list, st_kb);
  if (i1 >= ns) return i1;
  const int plane_len = nk[1] * nk[2];
  const int last_plane = hk[i1 - 1] / plane_len;
  if (hk[i1] / plane_len != last_plane || hk[i0] / plane_len == last_plane) return i1;  // already on a boundary
  int64_t cut = i1;
  while (cut > i0 && hk[cut - 1] / plane_len == last_plane) --cut;
  kb_list->clear();
  st_kb->clear();
  for (int64_t i = i0; i < cut; ++i) {
    if (kb_list->empty() || kb_list->back() != hk[i]) kb_list->push_back(hk[i]);
    st_kb->push_back((int)kb_list->size() - 1);
  }
  return cut;
}

// Stage 1 of one batch of whole k points on the tensor cores (Sec. 5.5 Eq. 71):
// X[kb] = sum_Re w e^{ik.Re} g(Re, .) by a GEMM, then T[s][Rp][sa][m] = sum_n X[kb(s)] U_k[n][b(s)]
// (FP32, physical scale) with the batch's max |T| in *tmaxp.  With Tb_out == nullptr the rotation
// is left to the caller: *X_out, *ldx_out receive the GEMM output (scaled by 1 / unscale).
template <int FMT, int NSPLIT, int NPROD>
static int stage1_batch(phoebe_gpu_ctx* c, const GridMap& gm, const std::vector<int>& kb_list,
                        const std::vector<int>& st_kb, int64_t i0, const int* st_k, const int* st_b, const cplx* UF,
                        const Parts& Pg, float sA1, const cplx* cis_k, const GridPhase& gk, int* err, unsigned* tmaxp,
                        const int* d_kb, const int* d_stkb, float2** Tb_out, const float** X_out = nullptr,
                        int64_t* ldx_out = nullptr) {
  const int nw = c->nw, nm = 3 * c->na, nRe = c->nRe, nRp = c->nRp;
  const int esz = FMT == 2 ? 4 : 2;
  const int KB = 128 / esz;
  const int Kp1 = (2 * nRe + KB - 1) / KB * KB;
  const int64_t C = (int64_t)nRp * nw * nw * nm;
  const int BN1 = StoreEpi::BN;
  const int S = (int)st_kb.size(), nkb = (int)kb_list.size();
  int st;
  const int64_t ldx = (2 * C + 3) / 4 * 4;  // row stride of X, 16-byte aligned
  Parts PAk;
  TRY(ensure_parts(c, "tc_Ak", NSPLIT, (size_t)nkb * Kp1, esz, &PAk));
  float* X = (float*)ensure(c, "tc_X", sizeof(float) * nkb * ldx, &st);
  if (!X) return st;
  {
    int64_t nt = (int64_t)nkb * (Kp1 / 2);
    k_pack_phase<FMT, NSPLIT><<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(
        d_kb, nkb, (const int*)c->bufs["Re"].p, (const double*)c->bufs["we"].p, nRe, gk, cis_k, Kp1, sA1, PAk);
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
    a.kb_per_chunk = PHX_KB_PER_CHUNK;
    a.b_row_step = BN1;
    a.group_m = std::max(1, a.m_tiles);
    a.ntiles = a.m_tiles * a.n_tiles;
    a.tile_list = nullptr;
    a.ntiles_dev = nullptr;
    a.err = err;
    StoreEpi::Params ep{X, ldx, nkb, (int)(2 * C)};
    TRY(launch_gemm<StoreEpi, FMT, NSPLIT, NPROD>(c, tAk, tG, a, ep));
  }
  if (!Tb_out) {
    *X_out = X;
    *ldx_out = ldx;
    return PHOEBE_GPU_OK;
  }
  float2* Tb = (float2*)ensure(c, "tc_T", sizeof(float2) * (size_t)S * nRp * nm * nw, &st);
  if (!Tb) return st;
  CK(c, cudaMemsetAsync(tmaxp, 0, 64, c->stream));
  {
    int64_t nt = (int64_t)S * nRp * nm * nw;
    const float unscale1 = 1.0f / (sA1 * c->tc->g_scale);
    k_pack_t<<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(X, ldx, unscale1, d_stkb, st_k + i0, st_b + i0,
                                                                   gm, UF, S, nRp, nw, nm, Tb, tmaxp);
    c->launches++;
    CK(c, cudaGetLastError());
  }
  *Tb_out = Tb;
  return PHOEBE_GPU_OK;
}

// Sampled q sums: stage 1 on the tensor cores per batch of whole k points, then the
// importance-sampled pairs of each batch (sampler.cu) in place of the full-grid stage 2.
template <int NW, int NM, int FMT, int NSPLIT, int NPROD>
static int run_sampled(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, const GridMap& gm, int64_t ns,
                       const std::vector<int>& hk, const int* st_k, const int* st_b, const double* epsF,
                       const double* fF, const cplx* UF, const double* omega, const double* nB, const cplx* Zq,
                       double* raw, const float2* UH, const float* f32, const float2* eps2, double omega_max,
                       const Parts& Pg, float sA1, const cplx* cis_k, const GridPhase& gk, int* err) {
  int st;
  Timer tm;
  IsTables it;
  it.epsF = epsF;
  it.fF = fF;
  it.UF = UF;
  it.eps2 = eps2;
  it.f32 = f32;
  it.UH = UH;
  it.omega = omega;
  it.nB = nB;
  it.Zq = Zq;
  it.omega_max = omega_max;
  unsigned* tmaxp = (unsigned*)ensure(c, "tc_tmax", 64, &st);
  if (!tmaxp) return st;
  // batches of whole k points: the proposal of a k mixes all its active bands
  const int max_states = p->max_batch_states > 0 ? p->max_batch_states : 1024;
  std::vector<int> kb_list, st_kb;
  int64_t i0 = 0;
  while (i0 < ns) {
    const int64_t i1 = next_batch(hk, ns, i0, max_states, &kb_list, &st_kb);
    const int S = (int)(i1 - i0);
    const int nkb = (int)kb_list.size();
    void *d_kb, *d_stkb;
    TRY(upload(c, "tc_batch_k", kb_list.data(), sizeof(int) * nkb, &d_kb));
    TRY(upload(c, "tc_batch_stkb", st_kb.data(), sizeof(int) * S, &d_stkb));
    tm.begin(c);
    float2* Tb;
    TRY((stage1_batch<FMT, NSPLIT, NPROD>(c, gm, kb_list, st_kb, i0, st_k, st_b, UF, Pg, sA1, cis_k, gk, err, tmaxp,
                                          (const int*)d_kb, (const int*)d_stkb, &Tb)));
    tm.end(c, &c->stats.stage1_ms);
    IsBatch ib;
    ib.S = S;
    ib.nkb = nkb;
    ib.s_base = i0;
    ib.st_k = st_k + i0;
    ib.st_b = st_b + i0;
    ib.st_kb = (const int*)d_stkb;
    ib.kb = (const int*)d_kb;
    ib.st_kb_host = &st_kb;
    ib.kb_host = &kb_list;
    ib.T = Tb;
    TRY(is_batch<NW, NM>(c, p, gm, ib, it, raw));
    i0 = i1;
  }
  int herr = 0;
  CK(c, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (herr) return fail(c, PHOEBE_GPU_ERR_TIMEOUT, "a tensor-core pipeline wait ran out; results discarded");
  return PHOEBE_GPU_OK;
}

// Plain GEMM into HBM with 256- or 128-column tiles.
template <int FMT, int NSPLIT, int NPROD>
static int launch_store(phoebe_gpu_ctx* c, int bn, const CUtensorMap* A, const CUtensorMap* B, TcGemmArgs a,
                        const StoreParams& ep) {
  if (bn == 128) return launch_gemm<StoreEpi128, FMT, NSPLIT, NPROD>(c, A, B, a, ep);
  return launch_gemm<StoreEpi, FMT, NSPLIT, NPROD>(c, A, B, a, ep);
}

// Stage 2 for any (nw, 3na): the R_p contraction G = P_q T runs as a plain tensor-core GEMM
// into HBM, one q chunk at a time, and k_elph_generic applies U_{k+q}^dagger, Z_q and the
// delta weights (Sec. 3.2 Eq. 13, Sec. 4.2 Eq. 29).  Exact: no screening.
template <int FMT, int NSPLIT, int NPROD>
static int run_tc_generic(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, const GridMap& gm, int64_t ns,
                          const std::vector<int>& hk, const int* st_k, const int* st_b, const double* epsF,
                          const cplx* UF, const double* fF, const double* omega, const double* nB, const cplx* Zq,
                          double* raw) {
  const int nw = c->nw, nm = 3 * c->na, nRe = c->nRe, nRp = c->nRp;
  if (nm > kGenericMaxModes) return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "at most %d modes", kGenericMaxModes);
  const int esz = FMT == 2 ? 4 : 2;
  const int KB = 128 / esz;
  const int Kp1 = (2 * nRe + KB - 1) / KB * KB, Kp2 = (2 * nRp + KB - 1) / KB * KB;
  const int64_t C = (int64_t)nRp * nw * nw * nm;
  const int64_t NF = (int64_t)gm.nf[0] * gm.nf[1] * gm.nf[2];
  const int64_t Nq = (int64_t)gm.nq[0] * gm.nq[1] * gm.nq[2];
  const int cps = 2 * nw * nm;
  int st;
  Timer tm;
  int* err = (int*)ensure(c, "tc_err", 64, &st);
  if (!err) return st;
  CK(c, cudaMemsetAsync(err, 0, 64, c->stream));
  const float sA1 = host_pow2_scale(c->we_max), sA2 = host_pow2_scale(c->wp_max);
  TRY((ensure_g_operand<FMT, NSPLIT>(c, C, Kp1, esz)));
  Parts Pg{{c->tc->g_part[0], c->tc->g_part[1], c->tc->g_part[2]}};
  // FP32 tables
  tm.begin(c);
  float2* UH = (float2*)ensure(c, "tc_UH", sizeof(float2) * NF * nw * nw, &st);
  if (!UH) return st;
  float* f32 = (float*)ensure(c, "tc_f32", sizeof(float) * NF * nw, &st);
  if (!f32) return st;
  float2* eps2 = (float2*)ensure(c, "tc_eps2", sizeof(float2) * NF * nw, &st);
  if (!eps2) return st;
  unsigned long long* dmax = (unsigned long long*)ensure(c, "tc_max", 64, &st);
  if (!dmax) return st;
  k_tables_el<<<(unsigned)((NF * nw * nw + 255) / 256), 256, 0, c->stream>>>(UF, fF, epsF, NF, nw, UH, f32, eps2);
  CK(c, cudaMemsetAsync(dmax, 0, 64, c->stream));
  k_absmax_f64<<<64, 256, 0, c->stream>>>(omega, Nq * nm, dmax);
  float2* Zf = (float2*)ensure(c, "tcg_Zf", sizeof(float2) * Nq * nm * nm, &st);
  if (!Zf) return st;
  float* omf = (float*)ensure(c, "tcg_omf", sizeof(float) * Nq * nm, &st);
  if (!omf) return st;
  float* nBf = (float*)ensure(c, "tcg_nBf", sizeof(float) * Nq * nm, &st);
  if (!nBf) return st;
  k_tables_ph<<<(unsigned)((Nq * nm * nm + 255) / 256), 256, 0, c->stream>>>(Zq, omega, nB, Nq, nm, Zf, omf, nBf);
  c->launches += 3;
  CK(c, cudaGetLastError());
  unsigned long long ombits = 0;
  CK(c, cudaMemcpyAsync(&ombits, dmax, sizeof(ombits), cudaMemcpyDeviceToHost, c->stream));
  // A operand: q phases in q order, rows padded to a multiple of 128
  GridPhase gq = make_phase(gm.nq), gk = make_phase(gm.nk);
  cplx *cis_q, *cis_k;
  TRY(cis_table(c, gq, "cis_q", &cis_q));
  TRY(cis_table(c, gk, "cis_k", &cis_k));
  const int64_t Mrows = (Nq + 127) / 128 * 128;
  std::vector<int> q_of_row((size_t)Mrows, -1);
  for (int64_t q = 0; q < Nq; ++q) q_of_row[(size_t)q] = (int)q;
  void* d_qrow;
  TRY(upload(c, "tcg_q_of_row", q_of_row.data(), sizeof(int) * Mrows, &d_qrow));
  Parts PAq;
  TRY(ensure_parts(c, "tc_Aq", NSPLIT, (size_t)Mrows * Kp2, esz, &PAq));
  {
    int64_t nt = Mrows * (Kp2 / 2);
    k_pack_phase<FMT, NSPLIT><<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(
        (const int*)d_qrow, Mrows, (const int*)c->bufs["Rp"].p, (const double*)c->bufs["wp"].p, nRp, gq, cis_q, Kp2,
        sA2, PAq);
    c->launches++;
    CK(c, cudaGetLastError());
  }
  CK(c, cudaStreamSynchronize(c->stream));
  double omega_max;
  memcpy(&omega_max, &ombits, sizeof(double));
  tm.end(c, &c->stats.stage1_ms);
  unsigned* tmaxp = (unsigned*)ensure(c, "tc_tmax", 64, &st);
  if (!tmaxp) return st;
  Deferred* df = c->defer;
  const int64_t g_budget = df ? df->g_budget : (int64_t)512 << 20;  // bytes of G per q chunk
  // a deferred call keeps every state in one batch: its recorded launches use the batch's buffers
  const int max_states =
      df ? (int)ns
         : p->max_batch_states > 0 ? p->max_batch_states
                                   : (int)std::max<int64_t>(1, std::min<int64_t>(4096, g_budget / (128 * 4 * cps)));
  std::vector<int> kb_list, st_kb;
  int64_t i0 = 0;
  while (i0 < ns) {
    const int64_t i1 = next_batch(hk, ns, i0, max_states, &kb_list, &st_kb);
    const int S = (int)(i1 - i0);
    const int nkb = (int)kb_list.size();
    void *d_kb, *d_stkb;
    TRY(upload(c, "tc_batch_k", kb_list.data(), sizeof(int) * nkb, &d_kb));
    TRY(upload(c, "tc_batch_stkb", st_kb.data(), sizeof(int) * S, &d_stkb));
    tm.begin(c);
    float2* Tb;
    TRY((stage1_batch<FMT, NSPLIT, NPROD>(c, gm, kb_list, st_kb, i0, st_k, st_b, UF, Pg, sA1, cis_k, gk, err, tmaxp,
                                          (const int*)d_kb, (const int*)d_stkb, &Tb)));
    const int64_t ncols = (int64_t)S * cps;
    Parts PB;
    TRY(ensure_parts(c, "tc_B2", NSPLIT, (size_t)ncols * Kp2, esz, &PB));
    for (int i = 0; i < NSPLIT; ++i) CK(c, cudaMemsetAsync(PB.p[i], 0, (size_t)ncols * Kp2 * esz, c->stream));
    {
      int64_t nt = (int64_t)S * nRp * nm * nw;
      k_split_t<FMT, NSPLIT><<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(Tb, S, nRp, nw, nm, Kp2, tmaxp, PB);
      c->launches++;
      CK(c, cudaGetLastError());
    }
    tm.end(c, &c->stats.stage1_ms);
    const int64_t ldg = (ncols + 3) / 4 * 4;  // row stride of G, 16-byte aligned
    const int64_t qc = std::max<int64_t>(128, std::min<int64_t>(Mrows, g_budget / (4 * ldg) / 128 * 128));
    float* G = (float*)ensure(c, "tcg_G", sizeof(float) * qc * ldg, &st);
    if (!G) return st;
    // GEMM arguments of the q chunk starting at row q0 for a tile width bn and K blocks per partial kb
    auto chunk_args = [&](int64_t q0, int bn, int kb, CUtensorMap* tA, CUtensorMap* tB, TcGemmArgs* a,
                          StoreParams* ep) -> int {
      const int64_t rows = std::min(qc, Mrows - q0);
      Parts PAc;
      for (int i = 0; i < 3; ++i)
        PAc.p[i] = PAq.p[i] ? static_cast<uint8_t*>(PAq.p[i]) + (size_t)q0 * Kp2 * esz : nullptr;
      TRY(part_maps(c, tA, PAc, NSPLIT, FMT, Kp2, rows, 128));
      TRY(part_maps(c, tB, PB, NSPLIT, FMT, Kp2, ncols, (uint32_t)bn));
      a->m_tiles = (int)(rows / 128);
      a->n_tiles = (int)((ncols + bn - 1) / bn);
      a->kblocks = Kp2 / KB;
      a->kb_per_chunk = kb;
      a->b_row_step = bn;
      a->group_m = std::min(a->m_tiles, 16);
      a->ntiles = a->m_tiles * a->n_tiles;
      a->tile_list = nullptr;
      a->ntiles_dev = nullptr;
      a->err = err;
      *ep = StoreParams{G, ldg, (int)rows, (int)ncols};
      return PHOEBE_GPU_OK;
    };
    int bn = StoreEpi::BN, kbc = PHX_KB_PER_CHUNK;
    const std::vector<int64_t> tune_key = {(int64_t)FMT, NSPLIT, NPROD, Kp2, ncols, Mrows, qc};
    const auto tuned = c->tuned_tiles.find(tune_key);
    if (df && df->autotune && tuned != c->tuned_tiles.end()) {  // tuned by an earlier call on this context
      bn = tuned->second.first;
      kbc = tuned->second.second;
    } else if (df && df->autotune) {
      // autotuner: time every (tile width, K blocks per partial) candidate on the first q chunk
      static const int cand_bn[2] = {128, 256}, cand_kb[3] = {1, 2, 4};
      cudaEvent_t e0, e1;
      CK(c, cudaEventCreate(&e0));
      CK(c, cudaEventCreate(&e1));
      float best = 1e30f;
      for (int ib = 0; ib < 2; ++ib)
        for (int ik = 0; ik < 3; ++ik) {
          CUtensorMap tA[3], tB[3];
          TcGemmArgs a;
          StoreParams ep;
          TRY(chunk_args(0, cand_bn[ib], cand_kb[ik], tA, tB, &a, &ep));
          TRY((launch_store<FMT, NSPLIT, NPROD>(c, cand_bn[ib], tA, tB, a, ep)));  // warm-up
          CK(c, cudaEventRecord(e0, c->stream));
          TRY((launch_store<FMT, NSPLIT, NPROD>(c, cand_bn[ib], tA, tB, a, ep)));
          CK(c, cudaEventRecord(e1, c->stream));
          CK(c, cudaEventSynchronize(e1));
          float ms = 0.f;
          CK(c, cudaEventElapsedTime(&ms, e0, e1));
          df->tune_ms[ib * 3 + ik] = ms;
          if (ms < best) {
            best = ms;
            bn = cand_bn[ib];
            kbc = cand_kb[ik];
          }
        }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      c->tuned_tiles[tune_key] = {bn, kbc};
    } else if (df) {
      if (df->bn) bn = df->bn;
      if (df->kb) kbc = df->kb;
    }
    if (df) {
      df->bn = bn;
      df->kb = kbc;
    }
    for (int64_t q0 = 0; q0 < Mrows; q0 += qc) {
      const int64_t rows = std::min(qc, Mrows - q0);
      CUtensorMap tA[3], tB[3];
      TcGemmArgs a;
      StoreParams ep;
      TRY(chunk_args(q0, bn, kbc, tA, tB, &a, &ep));
      ElphGenericArgs e;
      e.G = G;
      e.ldg = ldg;
      e.q_of_row = (const int*)d_qrow;
      e.row0 = q0;
      e.S = S;
      e.st_k = st_k + i0;
      e.st_b = st_b + i0;
      e.epsF = epsF;
      e.gm = gm;
      e.nw = nw;
      e.nm = nm;
      e.eps2 = eps2;
      e.f32 = f32;
      e.UH = UH;
      e.Zf = Zf;
      e.omf = omf;
      e.nBf = nBf;
      e.reach = (float)(omega_max + p->delta_cut_sigmas * p->sigma_eV) * 1.0001f;
      e.inv_sigma = (float)(1.0 / p->sigma_eV);
      e.cut2 = (float)(p->delta_cut_sigmas * p->delta_cut_sigmas);
      e.scale_base = (2.0 * kPi / (double)Nq) / (kSqrtPi * p->sigma_eV) / ((double)sA2 * (double)sA2);
      e.tmax = tmaxp;
      e.gamma = raw;
      e.s_base = i0;
      if (df) {
        struct Maps {
          CUtensorMap A[3], B[3];
        } mp;
        for (int i = 0; i < 3; ++i) {
          mp.A[i] = tA[i];
          mp.B[i] = tB[i];
        }
        df->ops.push_back([c, mp, a, ep, e, rows, bn]() -> int {
          TRY((launch_store<FMT, NSPLIT, NPROD>(c, bn, mp.A, mp.B, a, ep)));
          if (launch_elph_generic(c->stream, e, rows) != 0) {
            cudaGetLastError();
            return fail(c, PHOEBE_GPU_ERR_CUDA, "launch of the generic stage-2 epilogue failed");
          }
          c->launches++;
          return PHOEBE_GPU_OK;
        });
        c->stats.stage2_launches++;
        continue;
      }
      tm.begin(c);
      TRY((launch_store<FMT, NSPLIT, NPROD>(c, bn, tA, tB, a, ep)));
      c->stats.stage2_launches++;
      tm.end(c, &c->stats.stage2_ms);
      tm.begin(c);
      if (launch_elph_generic(c->stream, e, rows) != 0) {
        cudaGetLastError();
        return fail(c, PHOEBE_GPU_ERR_CUDA, "launch of the generic stage-2 epilogue failed");
      }
      c->launches++;
      tm.end(c, &c->stats.delta_ms);
    }
    i0 = i1;
  }
  c->stats.pairs_executed = ns * Nq;
  c->stats.stage2_flops = 8.0 * (double)ns * Nq * nRp * nw * nm;
  if (df) return PHOEBE_GPU_OK;  // the batch checks the wait flag after its launch
  int herr = 0;
  CK(c, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (herr) return fail(c, PHOEBE_GPU_ERR_TIMEOUT, "a tensor-core pipeline wait ran out; results discarded");
  return PHOEBE_GPU_OK;
}

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

  TRY((ensure_g_operand<FMT, NSPLIT>(c, C, Kp1, esz)));
  Parts Pg{{c->tc->g_part[0], c->tc->g_part[1], c->tc->g_part[2]}};

  // FP32 epilogue tables
  tm.begin(c);
  float2* UH = (float2*)ensure(c, "tc_UH", sizeof(float2) * NF * nw * nw, &st);
  if (!UH) return st;
  float* f32 = (float*)ensure(c, "tc_f32", sizeof(float) * NF * nw, &st);
  if (!f32) return st;
  float2* eps2 = (float2*)ensure(c, "tc_eps2", sizeof(float2) * NF * nw, &st);
  if (!eps2) return st;
  unsigned long long* dmax = (unsigned long long*)ensure(c, "tc_max", 64, &st);
  if (!dmax) return st;
  k_tables_el<<<(unsigned)((NF * nw * nw + 255) / 256), 256, 0, c->stream>>>(UF, fF, epsF, NF, nw, UH, f32,
                                                                             eps2);
  CK(c, cudaMemsetAsync(dmax, 0, 64, c->stream));
  k_absmax_f64<<<64, 256, 0, c->stream>>>(omega, Nq * nm, dmax);
  c->launches += 2;
  CK(c, cudaGetLastError());
  unsigned long long ombits = 0;
  CK(c, cudaMemcpyAsync(&ombits, dmax, sizeof(ombits), cudaMemcpyDeviceToHost, c->stream));

  // sampled q sums (learned or uniform proposal) replace the full-grid stage 2
  const bool sampled = c->isreq != nullptr;
  // stage-2 A operand: q phases, rows in compact q blocks padded to 128
  GridPhase gq = make_phase(gm.nq), gk = make_phase(gm.nk);
  cplx *cis_q, *cis_k;
  TRY(cis_table(c, gq, "cis_q", &cis_q));
  TRY(cis_table(c, gk, "cis_k", &cis_k));
  QBlocks qb;
  if (sampled) {
    CK(c, cudaStreamSynchronize(c->stream));
    double omega_max;
    memcpy(&omega_max, &ombits, sizeof(double));
    tm.end(c, &c->stats.stage1_ms);
    return run_sampled<NW, NM, FMT, NSPLIT, NPROD>(c, p, gm, ns, hk, st_k, st_b, epsF, fF, UF, omega, nB, Zq, raw,
                                                    UH, f32, eps2, omega_max, Pg, sA1, cis_k, gk, err);
  }
  {
    const int shape[3] = {4, 4, 8};
    for (int i = 0; i < 3; ++i) {
      qb.b[i] = std::min(shape[i], gm.nq[i]);
      qb.nb[i] = (gm.nq[i] + qb.b[i] - 1) / qb.b[i];
      qb.B[i] = qb.b[i] * gm.sq[i];
      qb.nbox[i] = (gm.nf[i] + qb.B[i] - 1) / qb.B[i];
    }
  }
  const int nblk = qb.nb[0] * qb.nb[1] * qb.nb[2];
  const int64_t Mrows = (int64_t)nblk * 128;
  {
    std::vector<int> q_of_row((size_t)Mrows, -1);
    std::vector<int4> qinfo((size_t)Mrows, make_int4(0, 0, 0, -1));
    for (int blk = 0; blk < nblk; ++blk) {
      int bc[3];
      grid_coords(blk, qb.nb, bc);
      int r = 0;
      for (int x = 0; x < qb.b[0]; ++x)
        for (int y = 0; y < qb.b[1]; ++y)
          for (int z = 0; z < qb.b[2]; ++z, ++r) {
            int qc3[3] = {bc[0] * qb.b[0] + x, bc[1] * qb.b[1] + y, bc[2] * qb.b[2] + z};
            if (qc3[0] < gm.nq[0] && qc3[1] < gm.nq[1] && qc3[2] < gm.nq[2]) {
              const int q = (int)grid_flat(qc3, gm.nq);
              q_of_row[(size_t)blk * 128 + r] = q;
              qinfo[(size_t)blk * 128 + r] =
                  make_int4(qc3[0] * gm.sq[0], qc3[1] * gm.sq[1], qc3[2] * gm.sq[2], q);
            }
          }
    }
    void* d;
    TRY(upload(c, "tc_q_of_row", q_of_row.data(), sizeof(int) * Mrows, &d));
    TRY(upload(c, "tc_qinfo", qinfo.data(), sizeof(int4) * Mrows, &d));
  }
  const int* q_of_row_d = (const int*)c->bufs["tc_q_of_row"].p;
  const int4* qinfo_d = (const int4*)c->bufs["tc_qinfo"].p;
  float2* Zr = (float2*)ensure(c, "tc_Zr", sizeof(float2) * Mrows * nm * nm, &st);
  if (!Zr) return st;
  float* omr = (float*)ensure(c, "tc_omr", sizeof(float) * Mrows * nm, &st);
  if (!omr) return st;
  float* nBr = (float*)ensure(c, "tc_nBr", sizeof(float) * Mrows * nm, &st);
  if (!nBr) return st;
  k_tables_ph_rows<<<(unsigned)((Mrows * nm * nm + 255) / 256), 256, 0, c->stream>>>(Zq, omega, nB, q_of_row_d, Mrows,
                                                                                     nm, Zr, omr, nBr);
  c->launches++;
  CK(c, cudaGetLastError());
  Parts PAq;
  TRY(ensure_parts(c, "tc_Aq", NSPLIT, (size_t)Mrows * Kp2, esz, &PAq));
  {
    int64_t nt = Mrows * (Kp2 / 2);
    k_pack_phase<FMT, NSPLIT><<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(
        q_of_row_d, Mrows, (const int*)c->bufs["Rp"].p, (const double*)c->bufs["wp"].p, nRp, gq, cis_q, Kp2, sA2, PAq);
    c->launches++;
    CK(c, cudaGetLastError());
  }
  // band-energy bounds of the F-grid boxes matching the q blocks
  const int64_t nbox = (int64_t)qb.nbox[0] * qb.nbox[1] * qb.nbox[2];
  double* box_lo = (double*)ensure(c, "tc_box_lo", sizeof(double) * nbox * nw, &st);
  if (!box_lo) return st;
  double* box_hi = (double*)ensure(c, "tc_box_hi", sizeof(double) * nbox * nw, &st);
  if (!box_hi) return st;
  k_box_bounds<<<(unsigned)((nbox * nw + 127) / 128), 128, 0, c->stream>>>(epsF, gm, nw, qb, box_lo, box_hi);
  unsigned long long* exec_pairs = (unsigned long long*)ensure(c, "tc_exec_pairs", 64, &st);
  if (!exec_pairs) return st;
  CK(c, cudaMemsetAsync(exec_pairs, 0, 64, c->stream));
  c->launches++;
  CK(c, cudaGetLastError());
  CK(c, cudaStreamSynchronize(c->stream));
  double omega_max;
  memcpy(&omega_max, &ombits, sizeof(double));
  const double reach = omega_max + p->delta_cut_sigmas * p->sigma_eV;
  tm.end(c, &c->stats.stage1_ms);
  CUtensorMap tAq[3];
  TRY(part_maps(c, tAq, PAq, NSPLIT, FMT, Kp2, Mrows, 128));

  // stage-2 tiling: whole states per n tile
  using EE = ElphEpi<NW, NM>;
  const int cps = EE::CPS, spt = EE::SPT;
  const int BN1 = StoreEpi::BN, BN2 = EE::BN;
  const int kb_chunk = PHX_KB_PER_CHUNK;
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
    const int64_t ldx = (2 * C + 3) / 4 * 4;  // row stride of X, 16-byte aligned
    Parts PAk;
    TRY(ensure_parts(c, "tc_Ak", NSPLIT, (size_t)nkb * Kp1, esz, &PAk));
    float* X = (float*)ensure(c, "tc_X", sizeof(float) * nkb * ldx, &st);
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
      a.tile_list = nullptr;
      a.ntiles_dev = nullptr;
      a.err = err;
      StoreEpi::Params ep{X, ldx, nkb, (int)(2 * C)};
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
      k_pack_t<<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(X, ldx, unscale1, (const int*)d_stkb, st_k + i0,
                                                                     st_b + i0, gm, UF, S, nRp, nw, nm, Tb, tmaxp);
      k_split_t<FMT, NSPLIT><<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(Tb, S, nRp, nw, nm, Kp2, tmaxp, PB);
      c->launches += 2;
      CK(c, cudaGetLastError());
    }
    tm.end(c, &c->stats.stage1_ms);

    // ---- screening: (q block, state) pairs that can contribute, compacted into a tile list
    tm.begin(c);
    const int n_tiles2 = (S + spt - 1) / spt;
    const int group_m2 = std::min(nblk, 64);
    const int64_t dense = (int64_t)nblk * n_tiles2;
    unsigned char* flag = (unsigned char*)ensure(c, "tc_flag", (size_t)S * nblk, &st);
    if (!flag) return st;
    int* tflag = (int*)ensure(c, "tc_tflag", sizeof(int) * dense, &st);
    if (!tflag) return st;
    int64_t* toff = (int64_t*)ensure(c, "tc_toff", sizeof(int64_t) * (dense + 1), &st);
    if (!toff) return st;
    int2* tlist = (int2*)ensure(c, "tc_tlist", sizeof(int2) * dense, &st);
    if (!tlist) return st;
    k_screen<<<(unsigned)(((int64_t)S * nblk + 127) / 128), 128, 0, c->stream>>>(
        st_k + i0, st_b + i0, S, epsF, gm, nw, qb, box_lo, box_hi, reach, flag);
    k_tile_flags<<<(unsigned)((dense + 255) / 256), 256, 0, c->stream>>>(flag, S, nblk, spt, group_m2, nblk,
                                                                           n_tiles2, tflag);
    k_scan_single_block<<<1, 1024, 0, c->stream>>>(tflag, dense, toff);
    k_tile_write<<<(unsigned)((dense + 255) / 256), 256, 0, c->stream>>>(
        tflag, toff, S, spt, group_m2, nblk, n_tiles2, qb, gm.nq[0], gm.nq[1], gm.nq[2], tlist, exec_pairs);
    c->launches += 4;
    CK(c, cudaGetLastError());
    tm.end(c, &c->stats.window_ms);

    int4* sinfo = (int4*)ensure(c, "tc_sinfo", sizeof(int4) * S, &st);
    if (!sinfo) return st;
    double* seps = (double*)ensure(c, "tc_seps", sizeof(double) * S, &st);
    if (!seps) return st;
    k_state_info<<<(S + 127) / 128, 128, 0, c->stream>>>(st_k + i0, st_b + i0, S, gm, epsF, nw, sinfo, seps);
    c->launches++;
    CK(c, cudaGetLastError());

    // ---- stage 2 with the fused el-ph epilogue over the screened tiles
    CUtensorMap tB[3];
    TRY(part_maps(c, tB, PB, NSPLIT, FMT, Kp2, rows2, BN2));
    tm.begin(c);
    {
      TcGemmArgs a;
      a.m_tiles = nblk;
      a.n_tiles = n_tiles2;
      a.kblocks = Kp2 / KB;
      a.kb_per_chunk = kb_chunk;
      a.b_row_step = spt * cps;
      a.group_m = group_m2;
      a.ntiles = (int)dense;
      a.tile_list = tlist;
      a.ntiles_dev = toff + dense;
      a.err = err;
      typename EE::Params ep;
      ep.Mq = (int)Mrows;
      ep.S = S;
      ep.sinfo = sinfo;
      ep.eps_n = seps;
      ep.s_base = i0;
      ep.gm = gm;
      ep.qinfo = qinfo_d;
      ep.eps2 = eps2;
      ep.fF = f32;
      ep.UH = UH;
      ep.Zr = Zr;
      ep.omr = omr;
      ep.nBr = nBr;
      ep.reach = (float)reach * 1.0001f;
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
  unsigned long long executed = 0;
  CK(c, cudaMemcpyAsync(&executed, exec_pairs, sizeof(executed), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->stats.pairs_executed = (int64_t)executed;
  c->stats.stage2_flops = 8.0 * (double)executed * nRp * nw * nm;  // executed algorithmic flops
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

// Stage 2 by the separable grid DFT (dft.cu): stage 1 in split FP16 on the tensor cores, then the
// R_p sum for every q of the grid in FP32 on the CUDA cores, with the fused rotations and deltas.
// Separable stage 1 of the grid-DFT mode (csrc/dft_s1.cu): residue tables of R_e on the k grid,
// the FP32 copy of g, phase tables.  *ok = false (and PHOEBE_GPU_OK) when the R_e set does not fit
// the kernel (more than 16 z groups or too much shared memory): the caller then takes the GEMM.
// With a64 != nullptr the FP64 form: g read in complex128, FP64 weights and phase tables in *a64.
static int s1_setup(phoebe_gpu_ctx* c, const GridMap& gm, S1Args* a, bool* ok, S64Args* a64 = nullptr) {
  *ok = false;
  const int nRe = c->nRe, nw = c->nw, nm = 3 * c->na;
  const int64_t C = (int64_t)c->nRp * nw * nw * nm;
  const int N3[3] = {gm.nk[0], gm.nk[1], gm.nk[2]};
  std::vector<int> Re((size_t)3 * nRe);
  std::vector<double> we(nRe);
  CK(c, cudaMemcpyAsync(Re.data(), c->bufs["Re"].p, sizeof(int) * 3 * nRe, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(we.data(), c->bufs["we"].p, sizeof(double) * nRe, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  std::vector<int> res[3], idx((size_t)3 * nRe);
  for (int d = 0; d < 3; ++d) {
    std::vector<int> r(nRe);
    for (int i = 0; i < nRe; ++i) r[i] = ((Re[3 * i + d] % N3[d]) + N3[d]) % N3[d];
    res[d] = r;
    std::sort(res[d].begin(), res[d].end());
    res[d].erase(std::unique(res[d].begin(), res[d].end()), res[d].end());
    for (int i = 0; i < nRe; ++i)
      idx[3 * i + d] = (int)(std::lower_bound(res[d].begin(), res[d].end(), r[i]) - res[d].begin());
  }
  const int Bx = (int)res[0].size(), By = (int)res[1].size(), Bz = (int)res[2].size();
  // entries sorted by (rz, ry, rx) residue index; pairs = distinct (rz, ry)
  std::vector<int> order(nRe);
  for (int i = 0; i < nRe; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int p, int q) {
    for (int d = 2; d >= 0; --d)
      if (idx[3 * p + d] != idx[3 * q + d]) return idx[3 * p + d] < idx[3 * q + d];
    return p < q;
  });
  std::vector<int> ent_row(nRe), ent_ax(nRe), peo, pay, rzo(Bz + 1, 0);
  std::vector<float> ent_w(nRe);
  for (int e = 0; e < nRe; ++e) {
    const int r = order[e];
    ent_row[e] = r;
    ent_ax[e] = idx[3 * r];
    ent_w[e] = (float)we[r];
    if (e == 0 || idx[3 * r + 1] != idx[3 * order[e - 1] + 1] || idx[3 * r + 2] != idx[3 * order[e - 1] + 2]) {
      peo.push_back(e);
      pay.push_back(idx[3 * r + 1]);
    }
    rzo[idx[3 * r + 2] + 1] = (int)peo.size();
  }
  const int Pe = (int)pay.size();
  peo.push_back(nRe);
  for (int z = 1; z <= Bz; ++z) rzo[z] = std::max(rzo[z], rzo[z - 1]);
  // z groups {r, -r mod Nz}
  std::vector<int> zgrp, zres;
  std::vector<char> done(Bz, 0);
  for (int z = 0; z < Bz; ++z) {
    if (done[z]) continue;
    const int rn = (N3[2] - res[2][z]) % N3[2];
    const int zn = (int)(std::lower_bound(res[2].begin(), res[2].end(), rn) - res[2].begin());
    const bool partner = zn < Bz && zn != z && res[2][zn] == rn;
    done[z] = 1;
    if (partner) done[zn] = 1;
    zgrp.push_back(z);
    zgrp.push_back(partner ? zn : -1);
    zres.push_back(res[2][z]);
  }
  const int Gz = (int)zres.size();
  // y groups within each rz: the pairs whose ry residues are r and -r mod Ny; a residue equal to its
  // negative, or whose negative has no pair at this rz, forms a group with itself
  std::vector<int> ygrp, ygrp_ay, rzg(Bz + 1, 0);
  for (int z = 0; z < Bz; ++z) {
    for (int p = rzo[z]; p < rzo[z + 1]; ++p) {
      const int rn = (N3[1] - res[1][pay[p]]) % N3[1];
      int pn = p;
      for (int p2 = rzo[z]; p2 < rzo[z + 1]; ++p2)
        if (p2 != p && res[1][pay[p2]] == rn) pn = p2;
      if (pn < p) continue;  // listed with its partner
      ygrp.push_back(p);
      ygrp.push_back(pn);
      ygrp_ay.push_back(pay[p]);
    }
    rzg[z + 1] = (int)ygrp_ay.size();
  }
  const int Gy = (int)ygrp_ay.size();
  const size_t s1_smem = a64 ? s64_smem_bytes(nRe, Pe, Bz, Gz, N3[1], By, N3[2])
                             : s1_smem_bytes(nRe, Pe, Bz, Gz, N3[1], By, N3[2], Gy);
  if (Gz > 16 || s1_smem > 200 * 1024 || (!a64 && 2 * C > INT32_MAX)) return PHOEBE_GPU_OK;  // the GEMM stage 1 serves
  int st;
  float2* g32 = nullptr;
  if (!a64) {
    g32 = (float2*)ensure(c, "s1_g32", sizeof(float2) * (size_t)nRe * C, &st);
    if (!g32) return st;
    if (s1_convert_g(c->stream, (const cplx*)c->bufs["g"].p, (int64_t)nRe * C, g32)) {
      cudaGetLastError();
      return fail(c, PHOEBE_GPU_ERR_CUDA, "launch of the stage-1 operand conversion failed");
    }
  }
  void *d_row, *d_ax, *d_w, *d_peo, *d_pay, *d_rzo, *d_zg, *d_rx, *d_ry, *d_rz;
  TRY(upload(c, "s1_row", ent_row.data(), sizeof(int) * nRe, &d_row));
  TRY(upload(c, "s1_ax", ent_ax.data(), sizeof(int) * nRe, &d_ax));
  TRY(upload(c, "s1_w", ent_w.data(), sizeof(float) * nRe, &d_w));
  TRY(upload(c, "s1_peo", peo.data(), sizeof(int) * (Pe + 1), &d_peo));
  TRY(upload(c, "s1_pay", pay.data(), sizeof(int) * Pe, &d_pay));
  TRY(upload(c, "s1_rzo", rzo.data(), sizeof(int) * (Bz + 1), &d_rzo));
  TRY(upload(c, "s1_zg", zgrp.data(), sizeof(int) * 2 * Gz, &d_zg));
  void *d_yg, *d_yay, *d_rzg;
  TRY(upload(c, "s1_yg", ygrp.data(), sizeof(int) * 2 * Gy, &d_yg));
  TRY(upload(c, "s1_yay", ygrp_ay.data(), sizeof(int) * Gy, &d_yay));
  TRY(upload(c, "s1_rzg", rzg.data(), sizeof(int) * (Bz + 1), &d_rzg));
  TRY(upload(c, "s1_rx", res[0].data(), sizeof(int) * Bx, &d_rx));
  TRY(upload(c, "s1_ry", res[1].data(), sizeof(int) * By, &d_ry));
  TRY(upload(c, "s1_rz", zres.data(), sizeof(int) * Gz, &d_rz));
  float2 *Ex = nullptr, *Ey = nullptr, *Ezg = nullptr;
  if (a64) {
    std::vector<double> wd(we.begin(), we.end());
    for (int e = 0; e < nRe; ++e) wd[e] = we[ent_row[e]];
    void* d_w64;
    TRY(upload(c, "s1_w64", wd.data(), sizeof(double) * nRe, &d_w64));
    double2* Ex64 = (double2*)ensure(c, "s1_Ex64", sizeof(double2) * N3[0] * Bx, &st);
    double2* Ey64 = Ex64 ? (double2*)ensure(c, "s1_Ey64", sizeof(double2) * N3[1] * By, &st) : nullptr;
    double2* Ez64 = Ey64 ? (double2*)ensure(c, "s1_Ezg64", sizeof(double2) * N3[2] * Gz, &st) : nullptr;
    if (!Ez64) return st;
    if (dft_table64(c->stream, (const int*)d_rx, Bx, N3[0], Ex64) ||
        dft_table64(c->stream, (const int*)d_ry, By, N3[1], Ey64) ||
        dft_table64(c->stream, (const int*)d_rz, Gz, N3[2], Ez64)) {
      cudaGetLastError();
      return fail(c, PHOEBE_GPU_ERR_CUDA, "launch of the FP64 stage-1 phase tables failed");
    }
    c->launches += 3;
    a64->g = (const double2*)c->bufs["g"].p;
    a64->ent_w = (const double*)d_w64;
    a64->Ex = Ex64;
    a64->Ey = Ey64;
    a64->Ezg = Ez64;
  } else {
    Ex = (float2*)ensure(c, "s1_Ex", sizeof(float2) * N3[0] * Bx, &st);
    Ey = Ex ? (float2*)ensure(c, "s1_Ey", sizeof(float2) * N3[1] * By, &st) : nullptr;
    Ezg = Ey ? (float2*)ensure(c, "s1_Ezg", sizeof(float2) * N3[2] * Gz, &st) : nullptr;
    if (!Ezg) return st;
    if (dft_table(c->stream, (const int*)d_rx, Bx, N3[0], Ex) ||
        dft_table(c->stream, (const int*)d_ry, By, N3[1], Ey) ||
        dft_table(c->stream, (const int*)d_rz, Gz, N3[2], Ezg)) {
      cudaGetLastError();
      return fail(c, PHOEBE_GPU_ERR_CUDA, "launch of the stage-1 phase tables failed");
    }
    c->launches += 4;
  }
  a->g = g32;
  a->C = C;
  a->nRe = nRe;
  a->Pe = Pe;
  a->Bx = Bx;
  a->By = By;
  a->Bz = Bz;
  a->Gz = Gz;
  a->nkx = N3[0];
  a->nky = N3[1];
  a->nkz = N3[2];
  a->ent_row = (const int*)d_row;
  a->ent_ax = (const int*)d_ax;
  a->ent_w = (const float*)d_w;
  a->pair_ent_off = (const int*)d_peo;
  a->pair_ay = (const int*)d_pay;
  a->rz_pair_off = (const int*)d_rzo;
  a->zgrp = (const int2*)d_zg;
  a->Gy = Gy;
  a->ygrp = (const int2*)d_yg;
  a->ygrp_ay = (const int*)d_yay;
  a->rz_grp_off = (const int*)d_rzg;
  a->Ex = Ex;
  a->Ey = Ey;
  a->Ezg = Ezg;
  if (a64) a64->i = *a;
  *ok = true;
  return PHOEBE_GPU_OK;
}

// X rows of one batch by the separable stage 1: the batch's k (kb_list, ascending grid indices;
// row = position in the list) grouped into kx planes and ky lines.  With a64 != nullptr the FP64
// form writes complex128 rows of C values to X64 (X and ldx unused).
static int s1_batch(phoebe_gpu_ctx* c, const GridMap& gm, S1Args a, const std::vector<int>& kb_list, float* X,
                    int64_t ldx, const S64Args* a64 = nullptr, double2* X64 = nullptr) {
  std::vector<int> pkx, ploff, lky, lkoff, kent;
  std::vector<std::pair<int, int>> line;  // (kz, row) of the current line
  const int nkz = gm.nk[2];
  auto flush = [&]() {  // entries of a line: k with its (-kz) partner when both are in the batch
    std::vector<int> row_of(nkz, -1);
    for (auto& e : line) row_of[e.first] = e.second;
    for (auto& e : line) {
      const int kz = e.first, kn = (nkz - kz) % nkz;
      if (kn != kz && row_of[kn] >= 0 && kn < kz) continue;  // taken with its partner
      kent.push_back(kz);
      kent.push_back(e.second);
      kent.push_back(kn != kz ? row_of[kn] : -1);
      kent.push_back(0);
    }
    line.clear();
  };
  int last_kx = -1, last_ky = -1;
  for (int i = 0; i < (int)kb_list.size(); ++i) {
    int kc[3];
    grid_coords(kb_list[i], gm.nk, kc);
    if (kc[0] != last_kx || kc[1] != last_ky) {
      flush();
      if (kc[0] != last_kx) {
        pkx.push_back(kc[0]);
        ploff.push_back((int)lky.size());
        last_kx = kc[0];
      }
      lky.push_back(kc[1]);
      lkoff.push_back((int)kent.size() / 4);
      last_ky = kc[1];
    }
    line.push_back({kc[2], i});
  }
  flush();
  const int planes = (int)pkx.size(), lines = (int)lky.size();
  ploff.push_back(lines);
  lkoff.push_back((int)kent.size() / 4);
  // one upload: kent (int4, first: 16-byte aligned), plane kx, plane line offsets, line ky, line k offsets
  std::vector<int> buf(kent);
  const size_t o1 = buf.size();
  buf.insert(buf.end(), pkx.begin(), pkx.end());
  const size_t o2 = buf.size();
  buf.insert(buf.end(), ploff.begin(), ploff.end());
  const size_t o3 = buf.size();
  buf.insert(buf.end(), lky.begin(), lky.end());
  const size_t o4 = buf.size();
  buf.insert(buf.end(), lkoff.begin(), lkoff.end());
  void* d;
  TRY(upload(c, "s1_batch", buf.data(), sizeof(int) * buf.size(), &d));
  const int* di = (const int*)d;
  a.X = X;
  a.ldx = ldx;
  a.kent = (const int4*)di;
  a.plane_kx = di + o1;
  a.plane_line_off = di + o2;
  a.line_ky = di + o3;
  a.line_k_off = di + o4;
  int r;
  if (a64) {
    S64Args b = *a64;
    b.i = a;
    b.X = X64;
    r = s64_launch(c->stream, b, planes);
  } else {
    r = s1_launch(c->stream, a, planes);
  }
  if (r) {
    cudaGetLastError();
    return fail(c, PHOEBE_GPU_ERR_CUDA, "launch of the separable stage 1 failed");
  }
  c->launches++;
  return PHOEBE_GPU_OK;
}

// fp64: the FP64 grid DFT (dft64.cu) with the same residue tables; every sum, table and Gaussian in
// FP64, the band and phonon arrays read as they are.
static int run_dft(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, const GridMap& gm, int64_t ns,
                   const std::vector<int>& hk, const int* st_k, const int* st_b, const double* epsF, const cplx* UF,
                   const double* fF, const double* omega, const double* nB, const cplx* Zq, double* raw,
                   bool fp64 = false) {
  constexpr int FMT = 0, NSPLIT = 2, NPROD = 3;
  const int nw = c->nw, nm = 3 * c->na, nRe = c->nRe, nRp = c->nRp;
  const int E = nw * nm;
  if (fp64 && (nw > 16 || nm > 30))
    return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "the FP64 grid DFT is built for nw <= 16 and 3na <= 30");
  if (!fp64 && !((nw == 1 || nw == 2 || nw == 4 || nw == 8) && (nm == 3 || nm == 6)))
    return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "the grid-DFT stage 2 is built for nw in {1, 2, 4, 8} and 3na in {3, 6}");
  const int Nx = gm.nq[0], Ny = gm.nq[1], Nz = gm.nq[2];
  if (Nx > 256)  // list entries hold jx in 8 bits
    return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "the grid-DFT stage 2 needs q-grid sizes Nx <= 256");
  const int esz = 2, KB = 64;
  const int Kp1 = (2 * nRe + KB - 1) / KB * KB;
  const int64_t C = (int64_t)nRp * nw * nw * nm;
  const int64_t NF = (int64_t)gm.nf[0] * gm.nf[1] * gm.nf[2];
  const int64_t Nq = (int64_t)Nx * Ny * Nz;
  int st;
  Timer tm;
  int* err = (int*)ensure(c, "tc_err", 64, &st);
  if (!err) return st;
  CK(c, cudaMemsetAsync(err, 0, 64, c->stream));
  unsigned long long* nq_eval = (unsigned long long*)ensure(c, "dft_nq_eval", 64, &st);
  if (!nq_eval) return st;
  CK(c, cudaMemsetAsync(nq_eval, 0, 64, c->stream));
  const float sA1 = host_pow2_scale(c->we_max);
  // stage 1 as a separable DFT over the R_e box when its tables fit, else the tensor-core GEMM
  S1Args s1a;
  S64Args s64a;
  bool s1_ok = false;
#ifndef PHX_S1_GEMM
  TRY(s1_setup(c, gm, &s1a, &s1_ok, fp64 ? &s64a : nullptr));
#endif
  if (fp64 && !s1_ok)
    return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "the FP64 grid DFT needs the R_e residue tables in shared memory");
  if (!s1_ok) TRY((ensure_g_operand<FMT, NSPLIT>(c, C, Kp1, esz)));
  Parts Pg{{nullptr, nullptr, nullptr}};  // the GEMM's operand parts (c->tc exists once they are built)
  if (!s1_ok) Pg = Parts{{c->tc->g_part[0], c->tc->g_part[1], c->tc->g_part[2]}};
  tm.begin(c);
  unsigned long long* dmax = (unsigned long long*)ensure(c, "tc_max", 64, &st);
  if (!dmax) return st;
  CK(c, cudaMemsetAsync(dmax, 0, 64, c->stream));
  k_absmax_f64<<<64, 256, 0, c->stream>>>(omega, Nq * nm, dmax);
  c->launches += 1;
  CK(c, cudaGetLastError());
  float2 *UH = nullptr, *ZT = nullptr, *omnb = nullptr;
  float* epsf = nullptr;
  float4* el4 = nullptr;
  if (!fp64) {  // FP32 tables of the FP32 kernels
    UH = (float2*)ensure(c, "tc_UH", sizeof(float2) * NF * nw * nw, &st);
    if (!UH) return st;
    float* f32 = (float*)ensure(c, "tc_f32", sizeof(float) * NF * nw, &st);
    if (!f32) return st;
    float2* eps2 = (float2*)ensure(c, "tc_eps2", sizeof(float2) * NF * nw, &st);
    if (!eps2) return st;
    epsf = (float*)ensure(c, "dft_epsf", sizeof(float) * NF * nw, &st);
    if (!epsf) return st;
    el4 = (float4*)ensure(c, "dft_el4", sizeof(float4) * NF * nw, &st);
    if (!el4) return st;
    ZT = (float2*)ensure(c, "dft_ZT", sizeof(float2) * Nq * nm * nm, &st);
    if (!ZT) return st;
    omnb = (float2*)ensure(c, "dft_omnb", sizeof(float2) * Nq * nm, &st);
    if (!omnb) return st;
    k_tables_el<<<(unsigned)((NF * nw * nw + 255) / 256), 256, 0, c->stream>>>(UF, fF, epsF, NF, nw, UH, f32, eps2);
    c->launches += 1;
    CK(c, cudaGetLastError());
    if (dft_tables(c->stream, epsF, fF, NF, nw, Zq, omega, nB, Nq, nm, epsf, el4, ZT, omnb)) {
      cudaGetLastError();
      return fail(c, PHOEBE_GPU_ERR_CUDA, "launch of the grid-DFT tables failed");
    }
    c->launches += 1;
  }
  float4* vel = nullptr;  // adaptive smearing: band velocities on the fine grid
  if (p->smearing == 1) TRY(velocity_grid(c, gm.nf, UF, &vel));
  float2* gL = nullptr;  // polar long-range term: L_{q nu} on the q grid
  if (c->have_polar) {
    gL = (float2*)ensure(c, "dft_gL", sizeof(float2) * Nq * nm, &st);
    if (!gL) return st;
    void* d_zs;
    TRY(upload(c, "polar_zstar", c->zstar.data(), sizeof(double) * 9 * c->na, &d_zs));
    PolarArgs pa;
    pa.zstar = (const double*)d_zs;
    pa.Zq = Zq;
    pa.out = gL;
    pa.Q = Nq;
    pa.na = c->na;
    pa.nm = nm;
    for (int d = 0; d < 3; ++d) pa.N[d] = gm.nq[d];
    const double* A = c->lattice;
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    const double inv[9] = {(A[4] * A[8] - A[5] * A[7]) / det, (A[2] * A[7] - A[1] * A[8]) / det,
                           (A[1] * A[5] - A[2] * A[4]) / det, (A[5] * A[6] - A[3] * A[8]) / det,
                           (A[0] * A[8] - A[2] * A[6]) / det, (A[2] * A[3] - A[0] * A[5]) / det,
                           (A[3] * A[7] - A[4] * A[6]) / det, (A[1] * A[6] - A[0] * A[7]) / det,
                           (A[0] * A[4] - A[1] * A[3]) / det};
    for (int i = 0; i < 3; ++i)  // b_i = 2 pi (row i of (A^-1)^T) = 2 pi (column i of A^-1)
      for (int cc = 0; cc < 3; ++cc) pa.B[3 * i + cc] = 2.0 * kPi * inv[3 * cc + i];
    for (int i = 0; i < 9; ++i) pa.eps[i] = c->eps_inf[i];
    pa.alpha = c->polar_alpha;
    pa.cut = 25.0;
    pa.pref = 4.0 * kPi / fabs(det) * kCoulombEVA;
    // G box: |q+G|^2 <= 4 alpha cut / lambda_min(eps) for every q of the first cell
    // smallest eigenvalue of the symmetric eps (trigonometric solution of the characteristic cubic)
    const double* ep = c->eps_inf;
    double lmin;
    {
      const double p1 = ep[1] * ep[1] + ep[2] * ep[2] + ep[5] * ep[5];
      if (p1 == 0.0) {
        lmin = std::min(ep[0], std::min(ep[4], ep[8]));
      } else {
        const double qm = (ep[0] + ep[4] + ep[8]) / 3.0;
        const double p2 = (ep[0] - qm) * (ep[0] - qm) + (ep[4] - qm) * (ep[4] - qm) + (ep[8] - qm) * (ep[8] - qm) +
                          2.0 * p1;
        const double pp = sqrt(p2 / 6.0);
        double Bm[9];
        for (int i = 0; i < 9; ++i) Bm[i] = (ep[i] - (i % 4 == 0 ? qm : 0.0)) / pp;
        const double r = 0.5 * (Bm[0] * (Bm[4] * Bm[8] - Bm[5] * Bm[7]) - Bm[1] * (Bm[3] * Bm[8] - Bm[5] * Bm[6]) +
                                Bm[2] * (Bm[3] * Bm[7] - Bm[4] * Bm[6]));
        const double phi = acos(std::max(-1.0, std::min(1.0, r))) / 3.0;
        lmin = qm + 2.0 * pp * cos(phi + 2.0 * kPi / 3.0);
      }
    }
    lmin *= 0.999;  // a bound: a slightly larger box is harmless
    const double kmax = sqrt(4.0 * pa.alpha * pa.cut / lmin);
    for (int i = 0; i < 3; ++i) {
      const double len = sqrt(A[3 * i] * A[3 * i] + A[3 * i + 1] * A[3 * i + 1] + A[3 * i + 2] * A[3 * i + 2]);
      pa.nmax[i] = (int)ceil(kmax / (2.0 * kPi) * len) + 1;
    }
    if (polar_table(c->stream, pa)) {
      cudaGetLastError();
      return fail(c, PHOEBE_GPU_ERR_CUDA, "launch of the polar long-range table failed");
    }
    c->launches++;
  }
  if (p->window_final == 1) {  // final-state window: excluded bands out of every reach
    k_final_window<<<(unsigned)((NF * nw + 255) / 256), 256, 0, c->stream>>>(
        epsF, NF * nw, p->mu_eV, p->window_eV, kBoltzmannEV * p->T_K, p->population_delta, epsf);
    c->launches++;
    CK(c, cudaGetLastError());
  }
  CK(c, cudaGetLastError());
  unsigned long long ombits = 0;
  CK(c, cudaMemcpyAsync(&ombits, dmax, sizeof(ombits), cudaMemcpyDeviceToHost, c->stream));
  // residues of R_p per axis and the entry lists of the y/z sums
  std::vector<int> Rp((size_t)3 * nRp);
  std::vector<double> wp(nRp);
  CK(c, cudaMemcpyAsync(Rp.data(), c->bufs["Rp"].p, sizeof(int) * 3 * nRp, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(wp.data(), c->bufs["wp"].p, sizeof(double) * nRp, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  const int N3[3] = {Nx, Ny, Nz};
  std::vector<int> resv[3];
  std::vector<int> idx((size_t)3 * nRp);
  for (int d = 0; d < 3; ++d) {
    std::vector<int> r(nRp);
    for (int i = 0; i < nRp; ++i) r[i] = ((Rp[3 * i + d] % N3[d]) + N3[d]) % N3[d];
    resv[d] = r;
    std::sort(resv[d].begin(), resv[d].end());
    resv[d].erase(std::unique(resv[d].begin(), resv[d].end()), resv[d].end());
    for (int i = 0; i < nRp; ++i)
      idx[3 * i + d] = (int)(std::lower_bound(resv[d].begin(), resv[d].end(), r[i]) - resv[d].begin());
  }
  const int Bx = (int)resv[0].size(), By = (int)resv[1].size(), Bz = (int)resv[2].size();
  // entries sorted by (rx, ry, rz) residue index; pairs = distinct (rx, ry); planes = distinct rx
  std::vector<int> order(nRp);
  for (int i = 0; i < nRp; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    for (int d = 0; d < 3; ++d)
      if (idx[3 * a + d] != idx[3 * b + d]) return idx[3 * a + d] < idx[3 * b + d];
    return a < b;
  });
  std::vector<int> plane_pair_off(Bx + 1, 0), pair_ent_off, pair_ay, ent_az(nRp), ent_r(nRp);
  for (int e = 0; e < nRp; ++e) {
    const int r = order[e];
    ent_az[e] = idx[3 * r + 2];
    ent_r[e] = r;
    const bool new_pair = e == 0 || idx[3 * r] != idx[3 * order[e - 1]] || idx[3 * r + 1] != idx[3 * order[e - 1] + 1];
    if (new_pair) {
      pair_ent_off.push_back(e);
      pair_ay.push_back(idx[3 * r + 1]);
    }
    plane_pair_off[idx[3 * r] + 1] = (int)pair_ent_off.size();
  }
  const int P = (int)pair_ay.size();
  pair_ent_off.push_back(nRp);
  for (int a = 1; a <= Bx; ++a) plane_pair_off[a] = std::max(plane_pair_off[a], plane_pair_off[a - 1]);
  int ne_plane_max = 0;
  for (int a = 0; a < Bx; ++a)
    ne_plane_max = std::max(ne_plane_max, pair_ent_off[plane_pair_off[a + 1]] - pair_ent_off[plane_pair_off[a]]);
  // x rows: each rx residue paired with its negative modulo Nx; a pair row carries S = Y_r + Y_-r and
  // D = Y_r - Y_-r.  Then the y groups of every x row: the ry residues present in its plane(s),
  // grouped as {r, -r mod Ny}, with the pair indices of the four combinations (P if absent).
  std::vector<int> xS, xD, xres;
  int K0 = 0, KP = 0;
  for (int pass = 0; pass < 3; ++pass) {  // real-factor rows, then pairs, then unpaired residues
    for (int a = 0; a < Bx; ++a) {
      const int r = resv[0][a], rn = (Nx - r) % Nx;
      const int b = (int)(std::lower_bound(resv[0].begin(), resv[0].end(), rn) - resv[0].begin());
      const bool has = b < Bx && resv[0][b] == rn;
      const int type = has && b == a ? 0 : has && b > a ? 1 : !has ? 2 : -1;
      if (type != pass) continue;
      xS.push_back(a);
      xD.push_back(type == 0 ? -1 : type == 1 ? b : a);
      xres.push_back(r);
      K0 += type == 0;
      KP += type == 1;
    }
  }
  const int K = (int)xS.size();
  std::vector<int> row_grp_off(1, 0), grp_idx, grp_ay;
  auto pair_of = [&](int plane, int ay) {
    for (int p = plane_pair_off[plane]; p < plane_pair_off[plane + 1]; ++p)
      if (pair_ay[p] == ay) return p;
    return P;
  };
  for (int k = 0; k < K; ++k) {
    const int a = xS[k], b = xD[k] >= 0 && xD[k] != xS[k] ? xD[k] : -1;
    std::vector<char> present(By, 0), done(By, 0);
    for (int pl : {a, b})
      if (pl >= 0)
        for (int p = plane_pair_off[pl]; p < plane_pair_off[pl + 1]; ++p) present[pair_ay[p]] = 1;
    for (int ay = 0; ay < By; ++ay) {
      if (!present[ay] || done[ay]) continue;
      const int rn = (Ny - resv[1][ay]) % Ny;
      const int an = (int)(std::lower_bound(resv[1].begin(), resv[1].end(), rn) - resv[1].begin());
      const bool partner = an < By && an != ay && resv[1][an] == rn && present[an];
      done[ay] = 1;
      if (partner) done[an] = 1;
      grp_idx.push_back(pair_of(a, ay));
      grp_idx.push_back(partner ? pair_of(a, an) : P);
      grp_idx.push_back(b >= 0 ? pair_of(b, ay) : P);
      grp_idx.push_back(b >= 0 && partner ? pair_of(b, an) : P);
      grp_ay.push_back(ay);
    }
    row_grp_off.push_back((int)grp_ay.size());
  }
  const int G = (int)grp_ay.size();
  const size_t smem_yx = fp64 ? dft64_smem_bytes(P, Bx, By, E, Nx, Ny, K, G) : dft_smem_bytes(P, Bx, By, nw, nm, Nx, Ny, K, G);
  const size_t smem_z = fp64 ? dft64_z_smem_bytes(ne_plane_max, E, Nz, Bz) : dft_z_smem_bytes(ne_plane_max, E, Nz, Bz);
  if (smem_yx > 227 * 1024 || smem_z > 227 * 1024)
    return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED,
                "the grid-DFT tiles (%d (rx, ry) residue pairs, Nx = %d) exceed shared memory", P, Nx);
  std::vector<float> wf(nRp);
  for (int i = 0; i < nRp; ++i) wf[i] = (float)wp[i];
  void *d_ppo, *d_peo, *d_az, *d_r, *d_w, *d_rx, *d_ry, *d_rz, *d_w64 = nullptr;
  if (fp64) TRY(upload(c, "dft_w64", wp.data(), sizeof(double) * nRp, &d_w64));
  TRY(upload(c, "dft_ppo", plane_pair_off.data(), sizeof(int) * (Bx + 1), &d_ppo));
  TRY(upload(c, "dft_peo", pair_ent_off.data(), sizeof(int) * (P + 1), &d_peo));
  void *d_gro, *d_gidx, *d_gay;
  TRY(upload(c, "dft_gro", row_grp_off.data(), sizeof(int) * (K + 1), &d_gro));
  TRY(upload(c, "dft_gidx", grp_idx.data(), sizeof(int) * 4 * std::max(G, 1), &d_gidx));
  TRY(upload(c, "dft_gay", grp_ay.data(), sizeof(int) * std::max(G, 1), &d_gay));
  TRY(upload(c, "dft_az", ent_az.data(), sizeof(int) * nRp, &d_az));
  TRY(upload(c, "dft_r", ent_r.data(), sizeof(int) * nRp, &d_r));
  TRY(upload(c, "dft_w", wf.data(), sizeof(float) * nRp, &d_w));
  void *d_xS, *d_xD;
  TRY(upload(c, "dft_rx", xres.data(), sizeof(int) * K, &d_rx));
  TRY(upload(c, "dft_xS", xS.data(), sizeof(int) * K, &d_xS));
  TRY(upload(c, "dft_xD", xD.data(), sizeof(int) * K, &d_xD));
  TRY(upload(c, "dft_ry", resv[1].data(), sizeof(int) * By, &d_ry));
  TRY(upload(c, "dft_rz", resv[2].data(), sizeof(int) * Bz, &d_rz));
  float2 *Ex = nullptr, *Ey = nullptr, *Ez = nullptr;
  double2 *Ex64 = nullptr, *Ey64 = nullptr, *Ez64 = nullptr;
  if (fp64) {
    Ex64 = (double2*)ensure(c, "dft_Ex64", sizeof(double2) * Nx * K, &st);
    if (!Ex64) return st;
    Ey64 = (double2*)ensure(c, "dft_Ey64", sizeof(double2) * Ny * By, &st);
    if (!Ey64) return st;
    Ez64 = (double2*)ensure(c, "dft_Ez64", sizeof(double2) * Nz * Bz, &st);
    if (!Ez64) return st;
    if (dft_table64(c->stream, (const int*)d_rx, K, Nx, Ex64) || dft_table64(c->stream, (const int*)d_ry, By, Ny, Ey64) ||
        dft_table64(c->stream, (const int*)d_rz, Bz, Nz, Ez64)) {
      cudaGetLastError();
      return fail(c, PHOEBE_GPU_ERR_CUDA, "launch of the FP64 DFT phase tables failed");
    }
  } else {
    Ex = (float2*)ensure(c, "dft_Ex", sizeof(float2) * Nx * K, &st);
    if (!Ex) return st;
    Ey = (float2*)ensure(c, "dft_Ey", sizeof(float2) * Ny * By, &st);
    if (!Ey) return st;
    Ez = (float2*)ensure(c, "dft_Ez", sizeof(float2) * Nz * Bz, &st);
    if (!Ez) return st;
    if (dft_table(c->stream, (const int*)d_rx, K, Nx, Ex) || dft_table(c->stream, (const int*)d_ry, By, Ny, Ey) ||
        dft_table(c->stream, (const int*)d_rz, Bz, Nz, Ez)) {
      cudaGetLastError();
      return fail(c, PHOEBE_GPU_ERR_CUDA, "launch of the DFT phase tables failed");
    }
  }
  c->launches += 3;
  GridPhase gk = make_phase(gm.nk);
  cplx* cis_k;
  TRY(cis_table(c, gk, "cis_k", &cis_k));
  double omega_max;
  memcpy(&omega_max, &ombits, sizeof(double));
  tm.end(c, &c->stats.stage1_ms);
  unsigned* tmaxp = (unsigned*)ensure(c, "tc_tmax", 64, &st);
  if (!tmaxp) return st;
  const int64_t per_state = (int64_t)P * Nz * E * (int64_t)(fp64 ? sizeof(double2) : sizeof(float2));
  const int max_states = p->max_batch_states > 0
                             ? std::min(p->max_batch_states, 65535)  // states run along gridDim.y
                             : (int)std::max<int64_t>(1, std::min<int64_t>(4096, ((int64_t)8 << 30) / per_state));
  std::vector<int> kb_list, st_kb;
  int64_t i0 = 0;
  while (i0 < ns) {
    const int64_t i1 = s1_ok ? next_batch_planes(hk, ns, i0, max_states, gm.nk, &kb_list, &st_kb)
                             : next_batch(hk, ns, i0, max_states, &kb_list, &st_kb);
    const int S = (int)(i1 - i0);
    const int nkb = (int)kb_list.size();
    void *d_kb, *d_stkb;
    TRY(upload(c, "tc_batch_k", kb_list.data(), sizeof(int) * nkb, &d_kb));
    TRY(upload(c, "tc_batch_stkb", st_kb.data(), sizeof(int) * S, &d_stkb));
    tm.begin(c);
    const float* X1 = nullptr;
    int64_t ldx1 = 0;
    double2* X64 = nullptr;
    if (fp64) {
      X64 = (double2*)ensure(c, "tc_X64", sizeof(double2) * (size_t)nkb * C, &st);
      if (!X64) return st;
      TRY(s1_batch(c, gm, s1a, kb_list, nullptr, 0, &s64a, X64));
    } else if (s1_ok) {
      ldx1 = (2 * C + 3) / 4 * 4;
      float* X = (float*)ensure(c, "tc_X", sizeof(float) * (size_t)nkb * ldx1, &st);
      if (!X) return st;
      TRY(s1_batch(c, gm, s1a, kb_list, X, ldx1));
      X1 = X;
    } else {
      TRY((stage1_batch<FMT, NSPLIT, NPROD>(c, gm, kb_list, st_kb, i0, st_k, st_b, UF, Pg, sA1, cis_k, gk, err, tmaxp,
                                            (const int*)d_kb, (const int*)d_stkb, nullptr, &X1, &ldx1)));
    }
    tm.end(c, &c->stats.stage1_ms);
    if (fp64) {
      double2* Zs64 = (double2*)ensure(c, "dft_Zs64", (size_t)per_state * S, &st);
      if (!Zs64) return st;
      DftZ64Args z;
      z.X = X64;
      z.ldx = C;
      z.st_kb = (const int*)d_stkb;
      z.st_k = st_k + i0;
      z.st_b = st_b + i0;
      z.gm = gm;
      z.UF = UF;
      z.nw = nw;
      z.w = (const double*)d_w64;
      z.nR = nRp;
      z.E = E;
      z.P = P;
      z.Nz = Nz;
      z.Bz = Bz;
      z.plane_pair_off = (const int*)d_ppo;
      z.pair_ent_off = (const int*)d_peo;
      z.ent_az = (const int*)d_az;
      z.ent_r = (const int*)d_r;
      z.Ez = Ez64;
      z.Zs = Zs64;
      DftX64Args x;
      x.Zs = Zs64;
      x.P = P;
      x.Bx = Bx;
      x.By = By;
      x.Nx = Nx;
      x.Ny = Ny;
      x.Nz = Nz;
      x.G = G;
      x.row_grp_off = (const int*)d_gro;
      x.grp_idx = (const int4*)d_gidx;
      x.grp_ay = (const int*)d_gay;
      x.K = K;
      x.K0 = K0;
      x.KP = KP;
      x.xS = (const int*)d_xS;
      x.xD = (const int*)d_xD;
      x.Ex = Ex64;
      x.Ey = Ey64;
      x.st_k = st_k + i0;
      x.st_b = st_b + i0;
      x.gm = gm;
      x.nw = nw;
      x.nm = nm;
      x.epsF = epsF;
      x.fF = fF;
      x.UF = UF;
      x.Zq = Zq;
      x.omega = omega;
      x.nB = nB;
      x.reach = (omega_max + p->delta_cut_sigmas * p->sigma_eV) * (1.0 + 1e-9);
      x.inv_sigma = 1.0 / p->sigma_eV;
      x.xcut = p->delta_cut_sigmas * p->sigma_eV;
      x.scale = (2.0 * kPi / (double)Nq) / (kSqrtPi * p->sigma_eV);
      x.gamma = raw;
      x.s_base = i0;
      x.nq_evaluated = nq_eval;
      tm.begin(c);
      if (dft64_launch(c->stream, z, x, S, ne_plane_max) != 0) {
        cudaGetLastError();
        return fail(c, PHOEBE_GPU_ERR_CUDA, "launch of the FP64 grid-DFT stage 2 failed");
      }
      c->launches += 2;
      c->stats.stage2_launches++;
      tm.end(c, &c->stats.stage2_ms);
      i0 = i1;
      continue;
    }
    float2* Zs = (float2*)ensure(c, "dft_Zs", (size_t)per_state * S, &st);
    if (!Zs) return st;
    DftZArgs zz;
    zz.X = X1;
    zz.ldx = ldx1;
    zz.unscale = s1_ok ? 1.0f : 1.0f / (sA1 * c->tc->g_scale);
    zz.st_kb = (const int*)d_stkb;
    zz.st_k = st_k + i0;
    zz.st_b = st_b + i0;
    zz.gm = gm;
    zz.UF = UF;
    zz.nw = nw;
    zz.w = (const float*)d_w;
    zz.nR = nRp;
    zz.E = E;
    zz.P = P;
    zz.Nz = Nz;
    zz.Bz = Bz;
    zz.plane_pair_off = (const int*)d_ppo;
    zz.pair_ent_off = (const int*)d_peo;
    zz.ent_az = (const int*)d_az;
    zz.ent_r = (const int*)d_r;
    zz.Ez = Ez;
    zz.Zs = Zs;
    DftXArgs x;
    x.Zs = Zs;
    x.P = P;
    x.Bx = Bx;
    x.By = By;
    x.Nx = Nx;
    x.Ny = Ny;
    x.Nz = Nz;
    x.G = G;
    x.row_grp_off = (const int*)d_gro;
    x.grp_idx = (const int4*)d_gidx;
    x.grp_ay = (const int*)d_gay;
    x.K = K;
    x.K0 = K0;
    x.KP = KP;
    x.xS = (const int*)d_xS;
    x.xD = (const int*)d_xD;
    x.Ex = Ex;
    x.Ey = Ey;
    x.st_k = st_k + i0;
    x.st_b = st_b + i0;
    x.epsF = epsF;
    x.gm = gm;
    x.epsf = epsf;
    x.el4 = el4;
    x.UH = UH;
    x.ZT = ZT;
    x.omnb = omnb;
    x.reach = (float)(omega_max + p->delta_cut_sigmas * p->sigma_eV) * 1.0001f;
    x.inv_sigma = (float)(1.0 / p->sigma_eV);
    x.cut2 = (float)(p->delta_cut_sigmas * p->delta_cut_sigmas);
    x.scale = (2.0 * kPi / (double)Nq) / (kSqrtPi * p->sigma_eV);
    x.gamma = raw;
    x.s_base = i0;
    x.nq_evaluated = nq_eval;
    x.err = err;
    x.pacc = c->prate_acc;
    x.mu = p->mu_eV;
    x.inv_kT = 1.0 / (kBoltzmannEV * p->T_K);
    x.vel = vel;
    x.gL = gL;
    x.UF = UF;
    x.sigma_min = (float)p->sigma_min_eV;
    x.omega_max = (float)omega_max;
    x.cut = (float)p->delta_cut_sigmas;
    for (int i = 0; i < 9; ++i) x.cB[i] = 0.f;
    if (vel) {  // cB[a][b] = (b_b)_a / N_b with b = 2 pi (A^-1)^T; the 1/sigma of each pair is in the sum
      const double* A = c->lattice;
      const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                         A[2] * (A[3] * A[7] - A[4] * A[6]);
      const double inv[9] = {(A[4] * A[8] - A[5] * A[7]) / det, (A[2] * A[7] - A[1] * A[8]) / det,
                             (A[1] * A[5] - A[2] * A[4]) / det, (A[5] * A[6] - A[3] * A[8]) / det,
                             (A[0] * A[8] - A[2] * A[6]) / det, (A[2] * A[3] - A[0] * A[5]) / det,
                             (A[3] * A[7] - A[4] * A[6]) / det, (A[1] * A[6] - A[0] * A[7]) / det,
                             (A[0] * A[4] - A[1] * A[3]) / det};  // inv[a][b] = (A^-1)_{ab}
      const int Nb[3] = {Nx, Ny, Nz};
      for (int a2 = 0; a2 < 3; ++a2)
        for (int b2 = 0; b2 < 3; ++b2) x.cB[a2 * 3 + b2] = (float)(2.0 * kPi * inv[a2 * 3 + b2] / Nb[b2]);
      x.scale = (2.0 * kPi / (double)Nq) / kSqrtPi;
    }
    tm.begin(c);
    const int r = dft_launch(c->stream, zz, x, S, nw, nm, ne_plane_max);
    if (r != 0) {
      cudaGetLastError();
      return fail(c, PHOEBE_GPU_ERR_CUDA, "launch of the grid-DFT stage 2 failed");
    }
    c->launches += 2;
    c->stats.stage2_launches++;
    tm.end(c, &c->stats.stage2_ms);
    i0 = i1;
  }
  int herr = 0;
  unsigned long long n_xb[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // four (pairs, bands) counters
  CK(c, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(n_xb, nq_eval, sizeof(n_xb), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  const unsigned long long n_x = n_xb[0] + n_xb[2] + n_xb[4] + n_xb[6], n_b = n_xb[1] + n_xb[3] + n_xb[5] + n_xb[7];
  if (herr) return fail(c, PHOEBE_GPU_ERR_TIMEOUT, "a pipeline wait of stage 1 or 2 ran out; results discarded");
  c->stats.pairs_executed = (int64_t)n_x;
  // complex MACs of the DFT: z sum over the entries, y sum over the pairs for every (jy, jz) line
  // (the lines a last, partial run of the fused kernel pads with are not counted), x sum per
  // evaluated (state, q)
  const double zy_cmac = ((double)nRp * Nz + (double)P * Ny * Nz) * E;
  // x sum: 4 FMA per complex value per residue pair or unpaired residue, 2 per real-factor residue
  double x_rows = 0.0;
  for (int k = 0; k < K; ++k) x_rows += xD[k] < 0 ? 0.5 : 1.0;
  // plus the epilogue's rotations U_{k+q}^dagger (nw x 3na complex MACs) and Z_q ((3na)^2) per listed
  // (state, q, band): counted exactly by the FP64 kernels, once per evaluated (state, q) by the FP32
  // ones (a lower bound: nearly every listed q has one band); the Gaussians and occupations are not
  // counted
  const double n_rot = fp64 ? (double)n_b : (double)n_x;
  c->stats.stage2_flops = 8.0 * ((double)ns * zy_cmac + (double)n_x * x_rows * E + n_rot * (E + nm * nm));
  return PHOEBE_GPU_OK;
}

static int run_tc_generic_mode(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, const GridMap& gm, int64_t ns,
                               const std::vector<int>& hk, const int* st_k, const int* st_b, const double* epsF,
                               const cplx* UF, const double* fF, const double* omega, const double* nB,
                               const cplx* Zq, double* raw) {
#define PHX_RUNG(FMT_, NS_, NP_) \
  return run_tc_generic<FMT_, NS_, NP_>(c, p, gm, ns, hk, st_k, st_b, epsF, UF, fF, omega, nB, Zq, raw)
  switch (p->precision) {
    case PHOEBE_PREC_SPLIT_BF16: PHX_RUNG(1, 3, 6);
    case PHOEBE_PREC_SPLIT_TF32: PHX_RUNG(2, 2, 3);
    case PHOEBE_PREC_BF16: PHX_RUNG(1, 1, 1);
    case PHOEBE_PREC_TF32: PHX_RUNG(2, 1, 1);
    case PHOEBE_PREC_SPLIT_FP16: PHX_RUNG(0, 2, 3);
    case PHOEBE_PREC_BF16X3: PHX_RUNG(1, 2, 3);
    default: return fail(c, PHOEBE_GPU_ERR_ARG, "unknown precision %d", p->precision);
  }
#undef PHX_RUNG
}

int run_tc(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, const GridMap& gm, int64_t ns,
           const std::vector<int>& hk, const int* st_k, const int* st_b, const double* epsF, const cplx* UF,
           const double* fF, const double* omega, const double* nB, const cplx* Zq, double* raw) {
  if (c->cc < 100) return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "tensor-core precisions need an sm_10x GPU");
  const int nw = c->nw, nm = 3 * c->na;
  if (p->precision == PHOEBE_PREC_FP32_DFT || p->precision == PHOEBE_PREC_FP64_DFT) {
    if (c->defer || c->isreq)
      return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "the grid-DFT stage 2 serves the full q sum of single calls");
    return run_dft(c, p, gm, ns, hk, st_k, st_b, epsF, UF, fF, omega, nB, Zq, raw,
                   p->precision == PHOEBE_PREC_FP64_DFT);
  }
  if (c->defer) {  // batched materials: one stage-2 form for every shape, recorded for later issue
    if (c->isreq) return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "batched linewidths use the full q sum");
    return run_tc_generic_mode(c, p, gm, ns, hk, st_k, st_b, epsF, UF, fF, omega, nB, Zq, raw);
  }
  if (nw == 8 && nm == 6) return run_tc_mode<8, 6>(c, p, gm, ns, hk, st_k, st_b, epsF, UF, fF, omega, nB, Zq, raw);
  if (nw == 2 && nm == 3) return run_tc_mode<2, 3>(c, p, gm, ns, hk, st_k, st_b, epsF, UF, fF, omega, nB, Zq, raw);
  if (nw == 1 && nm == 3) return run_tc_mode<1, 3>(c, p, gm, ns, hk, st_k, st_b, epsF, UF, fF, omega, nB, Zq, raw);
  if (c->isreq)
    return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED,
                "sampled q sums are built for (nw, 3na) in {(8,6), (2,3), (1,3)}; got (%d, %d)", nw, nm);
  return run_tc_generic_mode(c, p, gm, ns, hk, st_k, st_b, epsF, UF, fF, omega, nB, Zq, raw);
}

}  // namespace phx
