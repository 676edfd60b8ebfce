// Persistent warp-specialised tcgen05 GEMM for sm_103a.
//
// C[b] = alpha * A[b] * B[b]^T + beta * C[b] with A (M x K) and B (N x K)
// K-contiguous in global memory (BF16, or FP32 read as TF32); an operand may
// instead be MN-contiguous (A stored K x M, B stored K x N), in which case it
// is staged as MN-major tiles and the MMA reads it transposed.  Tiles of
// 128 x BN outputs are distributed over persistent CTAs; each CTA runs
//   warp 4      : TMA producer (one elected lane) filling a STAGES-deep ring
//                 of 128-byte-swizzled A/B slices, 128 bytes of K per slice;
//   warp 5      : TMEM allocator and MMA issuer (one elected lane), 4
//                 tcgen05.mma per slice into an FP32 accumulator in TMEM;
//   warps 0..3  : epilogue, tcgen05.ld of their 32-lane quadrant, alpha/beta,
//                 vector stores of C.
// Two TMEM accumulators (2 x BN columns) let the epilogue of tile i overlap
// the MMAs of tile i+1.  With GROUPED, the launch covers an uneven group of
// problems: the global tile index is mapped to (problem, tile) by binary
// search over the problems' first-tile offsets, and each problem brings its
// own tensor maps, C and K.
#pragma once
#include "common.cuh"
#include "tc_ptx.cuh"

namespace ks {
namespace tc {

struct TcArgs {
  int M, N, K, batch;
  int tiles_m, tiles_n, num_tiles, k_blocks;
  int raster;   // 0: consecutive tiles walk M (reuse the B slice), 1: walk N,
                // 2: groups of group_m tile rows, each walked along N (L2 locality)
  int group_m;  // raster 2: tile rows (units) per group, >= 1
  float alpha, beta;
  float* C;
  int64_t ldc, strideC;
  int vecC;
  int a_mn, b_mn;  // operand staged MN-major
  // Split-BF16 products: each operand holds nseg segments of seg_blocks
  // K-slices (its BF16 split parts, largest first) and segment g of the K'
  // loop multiplies A's part seg_map bits [2g, 2g + 2) by B's part seg_map bits
  // [16 + 2g, 16 + 2g + 2); seg_blocks is 0 for the other families.
  int seg_blocks, seg_map;
  int* status;
};

// One problem of a grouped launch, in device memory: its two tensor maps
// (128-byte aligned by their type, beyond the 64 bytes TMA requires), its C,
// and its first global tile index.
struct alignas(128) GroupDesc {
  CUtensorMap tmA;
  CUtensorMap tmB;
  float* C;
  int64_t ldc;
  int M, N, k_blocks, tiles_m, tiles_n, tile_start, vecC;
  int a_mn, b_mn, seg_blocks, seg_map;
  float alpha, beta;
};

struct GroupArgs {
  const GroupDesc* descs;
  int count;  // problems; descs[i].tile_start is ascending
};

constexpr int kThreads = 192;
constexpr int kBM = 128;

template <int BN, int STAGES, bool TF32>
struct TcCfg {
  static constexpr int ELEM = TF32 ? 4 : 2;
  static constexpr int BK = 128 / ELEM;        // K elements per slice (one 128-byte row)
  static constexpr int KMMA = TF32 ? 8 : 16;   // K per tcgen05.mma
  static constexpr int A_BYTES = kBM * 128;
  static constexpr int B_BYTES = BN * 128;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int TMEM_COLS = 2 * BN;     // 128, 256 or 512: power of two >= 32
  // Epilogue staging: 32 rows x 16 FP32 columns per epilogue warp.
  static constexpr int EPI_BYTES = 4 * 32 * 16 * 4;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + EPI_BYTES + 1024;
  // MN-major staging: one TMA box is MN_BOX MN elements (a 128-byte row) by
  // BK K rows; the boxes of a slice lie MN-block after MN-block.  The swizzle
  // atom is 8 K rows of one box for BF16 (128-byte swizzle, SBO 1 KB) and 4 K
  // rows for TF32 (128-byte swizzle of 32-byte pieces, SBO 512 bytes); the
  // descriptor steps one MN block by MN_BOX_BYTES (LBO), and each MMA's K range
  // starts KMMA rows (KMMA x 128 bytes) further on.
  static constexpr int MN_BOX = 128 / ELEM;
  static constexpr int MN_BOX_BYTES = BK * 128;
  static constexpr uint32_t MN_SBO = TF32 ? 512 : 1024;
  static constexpr uint32_t MN_MODE = TF32 ? kSw128Atom32 : kSw128;
};

__device__ __forceinline__ void tile_coords(const TcArgs& p, int tile, int& b, int& tm, int& tn) {
  const int per = p.tiles_m * p.tiles_n;
  b = tile / per;
  const int t = tile - b * per;
  if (p.raster == 2) {
    // Tile rows in groups of group_m (the last group may be shorter); inside a
    // group the index runs down the group's rows first, then along N, so the
    // tiles in flight at once share a few A and B slices that stay in L2.
    const int per_group = p.group_m * p.tiles_n;
    const int g = t / per_group;
    const int first = g * p.group_m;
    const int rows = min(p.group_m, p.tiles_m - first);
    const int r = t - g * per_group;
    tm = first + r % rows;
    tn = r / rows;
  } else if (p.raster == 0) {
    tm = t % p.tiles_m;
    tn = t / p.tiles_m;
  } else {
    tn = t % p.tiles_n;
    tm = t / p.tiles_n;
  }
}

// Where tile `tile` of the launch lives: operand maps, C and its geometry.
struct TileLoc {
  const CUtensorMap* ma;
  const CUtensorMap* mb;
  float* C;
  int64_t ldc, strideC;
  int M, N, k_blocks, b, tm, tn, vecC, a_mn, b_mn, seg_blocks, seg_map;
  float alpha, beta;
};

template <bool GROUPED>
__device__ __forceinline__ TileLoc locate(const TcArgs& p, const GroupArgs& g, const CUtensorMap* ma,
                                          const CUtensorMap* mb, int tile) {
  TileLoc L;
  if constexpr (GROUPED) {
    int lo = 0, hi = g.count - 1;  // last problem whose tile_start <= tile
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (g.descs[mid].tile_start <= tile) lo = mid; else hi = mid - 1;
    }
    const GroupDesc& d = g.descs[lo];
    const int t = tile - d.tile_start;
    L.ma = &d.tmA; L.mb = &d.tmB; L.C = d.C; L.ldc = d.ldc; L.strideC = 0;
    L.M = d.M; L.N = d.N; L.k_blocks = d.k_blocks; L.b = 0; L.vecC = d.vecC; L.a_mn = d.a_mn; L.b_mn = d.b_mn;
    L.seg_blocks = d.seg_blocks; L.seg_map = d.seg_map;
    L.alpha = d.alpha; L.beta = d.beta;
    if (p.raster == 0) { L.tm = t % d.tiles_m; L.tn = t / d.tiles_m; } else { L.tn = t % d.tiles_n; L.tm = t / d.tiles_n; }
  } else {
    L.ma = ma; L.mb = mb; L.C = p.C; L.ldc = p.ldc; L.strideC = p.strideC;
    L.M = p.M; L.N = p.N; L.k_blocks = p.k_blocks; L.vecC = p.vecC; L.alpha = p.alpha; L.beta = p.beta;
    L.a_mn = p.a_mn; L.b_mn = p.b_mn; L.seg_blocks = p.seg_blocks; L.seg_map = p.seg_map;
    tile_coords(p, tile, L.b, L.tm, L.tn);
  }
  return L;
}

// Stores one 32 x 32 chunk of C (rows row0 + lane of this warp's 32-row
// quadrant, columns n0 .. n0 + 31) from the registers of tcgen05.ld, where
// lane t holds row t.  Each 16-column half goes through this warp's 2 KB
// staging buffer (64-byte rows; the 16-byte piece q of row t sits at
// (t & 1) * 4 + (q ^ ((t >> 1) & 3)) within its 128-byte bank line, so both
// passes are free of bank conflicts) and is written back eight rows per
// instruction, each row a contiguous 64-byte run of C; beta != 0 reads C the
// same way.
__device__ __forceinline__ void store_chunk32(const TileLoc& p, float* cbase, int row0, int n0, float* stage,
                                              const uint32_t (&r)[32], int lane) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = 16 * h + 4 * q;
      const float4 v = make_float4(__uint_as_float(r[c]), __uint_as_float(r[c + 1]), __uint_as_float(r[c + 2]),
                                   __uint_as_float(r[c + 3]));
      *reinterpret_cast<float4*>(stage + lane * 16 + ((q ^ ((lane >> 1) & 3)) << 2)) = v;
    }
    __syncwarp();
    const int q = lane & 3, n = n0 + 16 * h + 4 * q;
#pragma unroll 2
    for (int i = 0; i < 4; ++i) {
      const int rr = 8 * i + (lane >> 2), row = row0 + rr;
      const float4 v = *reinterpret_cast<const float4*>(stage + rr * 16 + ((q ^ ((rr >> 1) & 3)) << 2));
      if (row >= p.M || n >= p.N) continue;
      float* crow = cbase + (int64_t)row * p.ldc;
      if (p.vecC && n + 3 < p.N) {
        float4 o = make_float4(p.alpha * v.x, p.alpha * v.y, p.alpha * v.z, p.alpha * v.w);
        if (p.beta != 0.f) {
          const float4 c = *reinterpret_cast<const float4*>(crow + n);
          o.x = fmaf(p.beta, c.x, o.x); o.y = fmaf(p.beta, c.y, o.y);
          o.z = fmaf(p.beta, c.z, o.z); o.w = fmaf(p.beta, c.w, o.w);
        }
        *reinterpret_cast<float4*>(crow + n) = o;
      } else {
        const float e4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (n + e < p.N) {
            float o = p.alpha * e4[e];
            if (p.beta != 0.f) o = fmaf(p.beta, crow[n + e], o);
            crow[n + e] = o;
          }
        }
      }
    }
    __syncwarp();  // the staging buffer is refilled by the next half
  }
}

template <int BN, int STAGES, bool TF32, bool GROUPED>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs p,
                   const GroupArgs g) {
  using Cfg = TcCfg<BN, STAGES, TF32>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], accf_bar[2], acce_bar[2];
  __shared__ uint32_t tmem_base_sh;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int unit0 = (int)blockIdx.x;
  const int units = (int)gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&accf_bar[a], 1);
      mbar_init(&acce_bar[a], 128);
    }
    fence_barrier_init();
  }
  if (!GROUPED && warp == 4 && lane == 0) {
    tma_prefetch(&tmA);
    tma_prefetch(&tmB);
  }
  if (warp == 5) tmem_alloc<Cfg::TMEM_COLS>(&tmem_base_sh);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_sh;
  // The prologue above (barriers, TMEM, tensor-map prefetch) touches no global
  // memory, so it may overlap the previous kernel's tail.
  pdl_wait();
  pdl_launch_dependents();

  if (warp == 4) {
    // ---------------------------------------------------------------- TMA producer
    if (elect_one()) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int tile = unit0; tile < p.num_tiles && ok; tile += units) {
        const TileLoc L = locate<GROUPED>(p, g, &tmA, &tmB, tile);
        for (int kb = 0; kb < L.k_blocks; ++kb) {
          if (!(ok = mbar_wait(&empty_bar[stage], phase ^ 1, p.status, kStatusTimeoutEmpty))) break;
          uint8_t* sa = smem + stage * Cfg::STAGE_BYTES;
          // K coordinates of this slice in A and B (split products: segment g
          // of the K' loop reads the parts of A and B that seg_map names).
          int xa = kb * Cfg::BK, xb = kb * Cfg::BK;
          if (!TF32 && L.seg_blocks > 0) {
            const int g = kb / L.seg_blocks, kk = kb - g * L.seg_blocks;
            xa = (((L.seg_map >> (2 * g)) & 3) * L.seg_blocks + kk) * Cfg::BK;
            xb = (((L.seg_map >> (16 + 2 * g)) & 3) * L.seg_blocks + kk) * Cfg::BK;
          }
          mbar_arrive_expect_tx(&full_bar[stage], Cfg::STAGE_BYTES);
          if (L.a_mn) {
#pragma unroll
            for (int j = 0; j < kBM / Cfg::MN_BOX; ++j)
              tma_load_3d(sa + j * Cfg::MN_BOX_BYTES, L.ma, &full_bar[stage], L.tm * kBM + j * Cfg::MN_BOX, xa,
                          L.b);
          } else {
            tma_load_3d(sa, L.ma, &full_bar[stage], xa, L.tm * kBM, L.b);
          }
          if (L.b_mn) {
#pragma unroll
            for (int j = 0; j < BN / Cfg::MN_BOX; ++j)
              tma_load_3d(sa + Cfg::A_BYTES + j * Cfg::MN_BOX_BYTES, L.mb, &full_bar[stage],
                          L.tn * BN + j * Cfg::MN_BOX, xb, L.b);
          } else {
            tma_load_3d(sa + Cfg::A_BYTES, L.mb, &full_bar[stage], xb, L.tn * BN, L.b);
          }
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      // Wait (bounded) until every issued slice has landed before the CTA can exit.
      if (ok) {
        for (int s = 0; s < STAGES; ++s) {
          if (!mbar_wait(&empty_bar[stage], phase ^ 1, p.status, kStatusTimeoutEmpty)) break;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
    }
  } else if (warp == 5) {
    // ---------------------------------------------------------------- MMA issuer
    if (elect_one()) {
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true;
      for (int tile = unit0; tile < p.num_tiles && ok; tile += units) {
        int k_blocks = p.k_blocks, a_mn = p.a_mn, b_mn = p.b_mn;
        if constexpr (GROUPED) {
          const TileLoc L = locate<true>(p, g, &tmA, &tmB, tile);
          k_blocks = L.k_blocks;
          a_mn = L.a_mn;
          b_mn = L.b_mn;
        }
        const uint32_t idesc = instr_desc<TF32>(kBM, BN, a_mn != 0, b_mn != 0);
        // K-major: the next MMA's K range starts KMMA elements along the swizzled
        // 128-byte row; MN-major: KMMA K rows further on, MN blocks MN_BOX_BYTES apart.
        const uint32_t a_step = a_mn ? Cfg::KMMA * 128 : Cfg::KMMA * Cfg::ELEM;
        const uint32_t b_step = b_mn ? Cfg::KMMA * 128 : Cfg::KMMA * Cfg::ELEM;
        const uint32_t a_lbo = a_mn ? Cfg::MN_BOX_BYTES : 16;
        const uint32_t b_lbo = b_mn ? Cfg::MN_BOX_BYTES : 16;
        if (!(ok = mbar_wait(&acce_bar[acc], acc_phase ^ 1, p.status, kStatusTimeoutAccEmpty))) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
        for (int kb = 0; kb < k_blocks; ++kb) {
          if (!(ok = mbar_wait(&full_bar[stage], phase, p.status, kStatusTimeoutFull))) break;
          tc_fence_after();
          const uint32_t a_addr = smem_u32(smem + stage * Cfg::STAGE_BYTES);
          const uint32_t b_addr = a_addr + Cfg::A_BYTES;
#pragma unroll
          for (int k = 0; k < Cfg::BK / Cfg::KMMA; ++k) {
            const uint64_t ad = a_mn ? smem_desc_sw128(a_addr + (uint32_t)k * a_step, a_lbo, Cfg::MN_SBO, Cfg::MN_MODE)
                                     : smem_desc_sw128(a_addr + (uint32_t)k * a_step, a_lbo, 1024);
            const uint64_t bd = b_mn ? smem_desc_sw128(b_addr + (uint32_t)k * b_step, b_lbo, Cfg::MN_SBO, Cfg::MN_MODE)
                                     : smem_desc_sw128(b_addr + (uint32_t)k * b_step, b_lbo, 1024);
            mma<TF32>(d_tmem, ad, bd, idesc, (kb | k) != 0 ? 1u : 0u);
          }
          mma_commit(&empty_bar[stage]);  // frees the slot once these MMAs have read it
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        mma_commit(&accf_bar[acc]);  // accumulator complete
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1;
        }
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 0..3)
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int tile = unit0; tile < p.num_tiles; tile += units) {
      if (!mbar_wait(&accf_bar[acc], acc_phase, p.status, kStatusTimeoutAcc)) break;
      tc_fence_after();
      const TileLoc L = locate<GROUPED>(p, g, &tmA, &tmB, tile);
      const int row0 = L.tm * kBM + warp * 32;
      float* cbase = L.C + (int64_t)L.b * L.strideC;
      float* stage = reinterpret_cast<float*>(smem + STAGES * Cfg::STAGE_BYTES) + warp * 32 * 16;
      const uint32_t tbase = tmem_base + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * BN);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        tmem_ld_32x32b_x32(tbase + (uint32_t)c0, r);
        tmem_ld_wait();
        if (row0 < L.M && L.tn * BN + c0 < L.N) store_chunk32(L, cbase, row0, L.tn * BN + c0, stage, r, lane);
      }
      tc_fence_before();
      mbar_arrive(&acce_bar[acc]);
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1;
      }
    }
  }

  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    tmem_dealloc<Cfg::TMEM_COLS>(tmem_base);
  }
}

}  // namespace tc
}  // namespace ks
