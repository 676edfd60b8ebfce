// FP32 SIMT GEMM family: the paper's parameterised tiled matrix multiply
// (Section 3) re-designed for sm_103a.
//
// Each thread owns a TM x TN register tile of C (the paper's R x C per work
// item); a WX x WY thread block covers a (WY*TM) x (WX*TN) tile; the K loop
// advances BK at a time.  Staged configs copy each BM x BK slice of op(A) and
// BK x BN slice of op(B) into a double-buffered shared-memory ring with
// coalesced 16-byte global loads (register prefetch of the next slice while the
// current one is consumed).  Unstaged configs read their operands straight
// from global memory with per-thread vector loads, as the paper's kernel does
// (it uses no local memory).  Threads own columns in 4-wide chunks spaced
// WX*4 apart (rows likewise), so shared-memory reads are conflict-free 16-byte
// loads and C stores form contiguous runs; for TN < 4 a warp-shuffle
// transpose regroups neighbouring threads' tiles into float4 stores.
#pragma once
#include <type_traits>
#include <utility>

#include "common.cuh"

namespace ks {

template <int TM_, int TN_, int WX_, int WY_, int BK_, bool STAGED_>
struct SimtCfg {
  static constexpr int TM = TM_, TN = TN_, WX = WX_, WY = WY_, BK = BK_;
  static constexpr bool STAGED = STAGED_;
  static constexpr int T = WX * WY;
  static constexpr int BM = WY * TM;
  static constexpr int BN = WX * TN;
  static constexpr int CM = TM < 4 ? TM : 4;  // contiguous rows per chunk
  static constexpr int CN = TN < 4 ? TN : 4;  // contiguous cols per chunk
  static constexpr int PAD = 4;
  static constexpr int LDS_A = BM + PAD;  // As[k][m]
  static constexpr int LDS_B = BN + PAD;  // Bs[k][n]
  static constexpr int STAGE_FLOATS = BK * (LDS_A + LDS_B);
  static constexpr int SMEM_BYTES = STAGED ? 2 * STAGE_FLOATS * 4 : 0;
  static constexpr int CHA = BM * BK / 4;  // 4-element chunks per slice
  static constexpr int CHB = BN * BK / 4;
  static constexpr int RA = (CHA + T - 1) / T;
  static constexpr int RB = (CHB + T - 1) / T;
  __device__ static constexpr int row(int i, int ty) { return (i / CM) * (WY * CM) + ty * CM + (i % CM); }
  __device__ static constexpr int col(int j, int tx) { return (j / CN) * (WX * CN) + tx * CN + (j % CN); }
  // Shared-memory position of column m of slice row k: the 4-float chunk index
  // is XORed with (k / 4) masked to the row's chunk count, which spreads the
  // transposing stores over the banks while every 4-aligned chunk stays
  // contiguous for the vector reads.
  __device__ static constexpr int swz_a(int m, int k) { return (((m >> 2) ^ ((k >> 2) & (BM / 4 - 1))) << 2) | (m & 3); }
  __device__ static constexpr int swz_b(int n, int k) { return (((n >> 2) ^ ((k >> 2) & (BN / 4 - 1))) << 2) | (n & 3); }
  // Lane that holds thread column tx ^ 1 of the same thread row (see thread_coords).
  static constexpr int TX_LANE_STRIDE = STAGED ? 2 : 1;
};

// Thread (tx, ty) of the WX x WY block that thread `tid` plays.  Unstaged configs
// read global memory directly and keep tx = tid % WX, so consecutive lanes read
// consecutive columns.  Staged configs read their fragments from shared memory,
// where the cost of a warp's load depends on which lanes share an address: a
// 16-byte load takes two wavefronts (one per half-warp) only when, in each half,
// its two quarter-warps touch disjoint banks or lanes sharing a chunk are
// neighbours (l, l ^ 1); otherwise four.  Each warp therefore covers 4 thread rows
// x 8 thread columns with the row in lane bit 0 (and bit 4) and the column in lane
// bits 1-3: the A fragment (per row) and the B fragment (per column) loads both
// meet the two-wavefront case (measured on GB300 with a per-pattern probe), where
// tx = tid % WX made every 16-byte B load take four.  Which thread owns which
// part of C is unchanged, so results are bit-identical.
template <class Cfg>
__device__ __forceinline__ void thread_coords(int tid, int& tx, int& ty) {
  if constexpr (Cfg::STAGED) {
    static_assert(Cfg::WX % 8 == 0 && Cfg::WY % 4 == 0, "lane map needs 8-column, 4-row warp blocks");
    const int w = tid >> 5, l = tid & 31;
    tx = (w % (Cfg::WX / 8)) * 8 + ((l >> 1) & 7);
    ty = (w / (Cfg::WX / 8)) * 4 + (((l >> 3) & 2) | (l & 1));
  } else {
    tx = tid % Cfg::WX;
    ty = tid / Cfg::WX;
  }
}

template <int W>
struct VecT;
template <>
struct VecT<1> { using T = float; };
template <>
struct VecT<2> { using T = float2; };
template <>
struct VecT<4> { using T = float4; };

template <int W>
__device__ __forceinline__ void load_vec_smem(float* dst, const float* src) {
  typename VecT<W>::T v = *reinterpret_cast<const typename VecT<W>::T*>(src);
  if constexpr (W == 1) {
    dst[0] = v;
  } else if constexpr (W == 2) {
    dst[0] = v.x; dst[1] = v.y;
  } else {
    dst[0] = v.x; dst[1] = v.y; dst[2] = v.z; dst[3] = v.w;
  }
}

// Global load of W consecutive floats at src[0..W) of operand `op`, element q
// valid when q < lim; one vector load when `vec` and all W are valid.
template <int W>
__device__ __forceinline__ void load_vec_global(float* dst, const float* src, int lim, bool vec, const GemmArgs& p,
                                                int op) {
  if (vec && lim >= W) {
    typename VecT<W>::T v = ks_in_bounds(p, op, src, 4 * W) ? __ldg(reinterpret_cast<const typename VecT<W>::T*>(src))
                                                             : typename VecT<W>::T{};
    if constexpr (W == 1) {
      dst[0] = v;
    } else if constexpr (W == 2) {
      dst[0] = v.x; dst[1] = v.y;
    } else {
      dst[0] = v.x; dst[1] = v.y; dst[2] = v.z; dst[3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < W; ++q) dst[q] = (q < lim && ks_in_bounds(p, op, src + q, 4)) ? __ldg(src + q) : 0.f;
  }
}

__device__ __forceinline__ float sel4(const float (&v)[4], int i) {
  return i == 0 ? v[0] : i == 1 ? v[1] : i == 2 ? v[2] : v[3];
}

// The TM x TN accumulator tile.  With TM even it is held as row pairs, so one
// packed FMA (__ffma2_rn: two FP32 FMAs, each rounded exactly like fmaf)
// updates rows i and i+1 of a column: the pair (a_i, a_i+1) arrives in
// consecutive registers from the vector shared-memory loads and b_j is
// duplicated once per column.  This halves the FMA instructions of the
// issue-bound inner loop without changing any result bit.
template <int TM, int TN>
struct AccTile {
  static constexpr bool PAIRED = (TM % 2 == 0);
  float2 v2[PAIRED ? TM / 2 : 1][TN];
  float v1[PAIRED ? 1 : TM][TN];

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int j = 0; j < TN; ++j) {
#pragma unroll
      for (int i = 0; i < (PAIRED ? TM / 2 : 1); ++i) v2[i][j] = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < (PAIRED ? 1 : TM); ++i) v1[i][j] = 0.f;
    }
  }
  __device__ __forceinline__ void fma(const float (&a)[TM], const float (&b)[TN]) {
    if constexpr (PAIRED) {
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const float2 bj = make_float2(b[j], b[j]);
#pragma unroll
        for (int i = 0; i < TM / 2; ++i) v2[i][j] = __ffma2_rn(make_float2(a[2 * i], a[2 * i + 1]), bj, v2[i][j]);
      }
    } else {
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) v1[i][j] = fmaf(a[i], b[j], v1[i][j]);
    }
  }
  __device__ __forceinline__ float get(int i, int j) const {
    if constexpr (PAIRED) return (i & 1) ? v2[i / 2][j].y : v2[i / 2][j].x;
    else return v1[i][j];
  }
};

template <class Cfg>
__device__ __forceinline__ void store_out(const GemmArgs& p, float* Cb, int gm, int gn, float v) {
  if (gm < p.M && gn < p.N) {
    float* dst = Cb + (int64_t)gm * p.ldc + gn;
    if (!ks_in_bounds(p, 2, dst, 4)) return;
    float out = p.alpha * v;
    if (p.beta != 0.f) out = fmaf(p.beta, *dst, out);
    *dst = out;
  }
}

// Four consecutive columns gn..gn+3 of row gm.
template <class Cfg>
__device__ __forceinline__ void store_out4(const GemmArgs& p, float* Cb, int gm, int gn, const float (&v)[4]) {
  if (gm >= p.M) return;
  float* dst = Cb + (int64_t)gm * p.ldc + gn;
  if (p.vecC && gn + 3 < p.N) {
    if (!ks_in_bounds(p, 2, dst, 16)) return;
    float4 o = make_float4(p.alpha * v[0], p.alpha * v[1], p.alpha * v[2], p.alpha * v[3]);
    if (p.beta != 0.f) {
      float4 c = *reinterpret_cast<const float4*>(dst);
      o.x = fmaf(p.beta, c.x, o.x); o.y = fmaf(p.beta, c.y, o.y);
      o.z = fmaf(p.beta, c.z, o.z); o.w = fmaf(p.beta, c.w, o.w);
    }
    *reinterpret_cast<float4*>(dst) = o;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) store_out<Cfg>(p, Cb, gm, gn + q, v[q]);
  }
}

template <class Cfg>
__device__ __forceinline__ void epilogue(const GemmArgs& p, float* Cb, int m0, int n0, int tx, int ty,
                                         const float (&acc)[Cfg::TM][Cfg::TN]) {
  constexpr int TM = Cfg::TM, TN = Cfg::TN, CN = Cfg::CN, XS = Cfg::TX_LANE_STRIDE;
  if constexpr (CN == 4) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int jc = 0; jc < TN / 4; ++jc) {
        float v[4] = {acc[i][jc * 4], acc[i][jc * 4 + 1], acc[i][jc * 4 + 2], acc[i][jc * 4 + 3]};
        store_out4<Cfg>(p, Cb, m0 + Cfg::row(i, ty), n0 + Cfg::col(jc * 4, tx), v);
      }
  } else if constexpr (CN == 2 && TM >= 2) {
    // Thread pairs (tx even/odd, XS lanes apart) hold columns 4g..4g+1 /
    // 4g+2..4g+3 of the same rows; swap half of each 2x4 block so each thread
    // owns one full row.
    const int q = tx & 1;
#pragma unroll
    for (int i0 = 0; i0 < TM; i0 += 2) {
      float s0 = q ? acc[i0][0] : acc[i0 + 1][0];
      float s1 = q ? acc[i0][1] : acc[i0 + 1][1];
      float r0 = __shfl_xor_sync(0xffffffffu, s0, XS);
      float r1 = __shfl_xor_sync(0xffffffffu, s1, XS);
      float v[4];
      if (q == 0) {
        v[0] = acc[i0][0]; v[1] = acc[i0][1]; v[2] = r0; v[3] = r1;
      } else {
        v[0] = r0; v[1] = r1; v[2] = acc[i0 + 1][0]; v[3] = acc[i0 + 1][1];
      }
      store_out4<Cfg>(p, Cb, m0 + Cfg::row(i0 + q, ty), n0 + (tx & ~1) * 2, v);
    }
  } else if constexpr (CN == 1 && TM >= 4) {
    // Thread quads (tx & 3, lanes XS apart) hold one column each of the same 4
    // rows: 4x4 transpose by butterfly shuffles so each thread owns one row of 4
    // columns.
    const int q = tx & 3;
#pragma unroll
    for (int i0 = 0; i0 < TM; i0 += 4) {
      float v[4] = {acc[i0][0], acc[i0 + 1][0], acc[i0 + 2][0], acc[i0 + 3][0]};
      // w[c] = element (row q, column c) of the 4x4 block; thread c of the quad holds column c.
      float w[4] = {q == 0 ? v[0] : 0.f, q == 1 ? v[1] : 0.f, q == 2 ? v[2] : 0.f, q == 3 ? v[3] : 0.f};
#pragma unroll
      for (int s = 1; s < 4; ++s) {
        float r = __shfl_xor_sync(0xffffffffu, sel4(v, q ^ s), s * XS);
        const int dst = q ^ s;
        w[0] = (dst == 0) ? r : w[0];
        w[1] = (dst == 1) ? r : w[1];
        w[2] = (dst == 2) ? r : w[2];
        w[3] = (dst == 3) ? r : w[3];
      }
      store_out4<Cfg>(p, Cb, m0 + Cfg::row(i0 + q, ty), n0 + (tx & ~3), w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) store_out<Cfg>(p, Cb, m0 + Cfg::row(i, ty), n0 + Cfg::col(j, tx), acc[i][j]);
  }
}

// ---------------------------------------------------------------- staged slice copy
// How a slice is read from global memory:
//   kLoadFast  : the whole slice lies inside op(A) / op(B) and 16-byte loads are
//                legal (interior tile, full K slice);
//   kLoadKTail : interior tile (rows and columns in range, 16-byte loads legal),
//                but the slice may run past K: only k is checked;
//   kLoadGeneral: every bound is checked (edge tiles, unaligned operands).
constexpr int kLoadGeneral = 0, kLoadKTail = 1, kLoadFast = 2;

template <class Cfg, int MODE>
__device__ __forceinline__ void load_slice_a(float4 (&r)[Cfg::RA], const GemmArgs& p, const float* Ab,
                                             int m0, int k0, int K, int tid) {
  constexpr int BK = Cfg::BK, BM = Cfg::BM;
#pragma unroll
  for (int u = 0; u < Cfg::RA; ++u) {
    const int c = tid + u * Cfg::T;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (c < Cfg::CHA) {
      if (!p.transA) {  // stored M x K: chunk of 4 along k
        const int m = c / (BK / 4), kq = (c % (BK / 4)) * 4;
        const int gm = m0 + m, gk = k0 + kq;
        const float* src = Ab + (int64_t)gm * p.lda + gk;
        if (MODE == kLoadFast) {
          r[u] = ks_in_bounds(p, 0, src, 16) ? __ldg(reinterpret_cast<const float4*>(src)) : float4{};
          continue;
        }
        if (MODE == kLoadKTail || gm < p.M) load_vec_global<4>(v, src, K - gk, MODE == kLoadKTail || p.vecA, p, 0);
      } else {  // stored K x M: chunk of 4 along m
        const int k = c / (BM / 4), mq = (c % (BM / 4)) * 4;
        const int gk = k0 + k, gm = m0 + mq;
        const float* src = Ab + (int64_t)gk * p.lda + gm;
        if (MODE == kLoadFast) {
          r[u] = ks_in_bounds(p, 0, src, 16) ? __ldg(reinterpret_cast<const float4*>(src)) : float4{};
          continue;
        }
        if (MODE == kLoadKTail) {
          r[u] = (gk < K && ks_in_bounds(p, 0, src, 16)) ? __ldg(reinterpret_cast<const float4*>(src)) : float4{};
          continue;
        }
        if (gk < K) load_vec_global<4>(v, src, p.M - gm, p.vecA, p, 0);
      }
    }
    r[u] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

template <class Cfg>
__device__ __forceinline__ void store_slice_a(const float4 (&r)[Cfg::RA], const GemmArgs& p, float* As, int tid) {
  constexpr int BK = Cfg::BK, BM = Cfg::BM, L = Cfg::LDS_A;
#pragma unroll
  for (int u = 0; u < Cfg::RA; ++u) {
    const int c = tid + u * Cfg::T;
    if (c < Cfg::CHA) {
      if (!p.transA) {
        const int m = c / (BK / 4), kq = (c % (BK / 4)) * 4;
        const int pm = Cfg::swz_a(m, kq);  // same chunk XOR for the 4 rows kq..kq+3
        As[(kq + 0) * L + pm] = r[u].x;
        As[(kq + 1) * L + pm] = r[u].y;
        As[(kq + 2) * L + pm] = r[u].z;
        As[(kq + 3) * L + pm] = r[u].w;
      } else {
        const int k = c / (BM / 4), mq = (c % (BM / 4)) * 4;
        *reinterpret_cast<float4*>(As + k * L + Cfg::swz_a(mq, k)) = r[u];
      }
    }
  }
}

template <class Cfg, int MODE>
__device__ __forceinline__ void load_slice_b(float4 (&r)[Cfg::RB], const GemmArgs& p, const float* Bb,
                                             int n0, int k0, int K, int tid) {
  constexpr int BK = Cfg::BK, BN = Cfg::BN;
#pragma unroll
  for (int u = 0; u < Cfg::RB; ++u) {
    const int c = tid + u * Cfg::T;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (c < Cfg::CHB) {
      if (!p.transB) {  // stored K x N: chunk along n
        const int k = c / (BN / 4), nq = (c % (BN / 4)) * 4;
        const int gk = k0 + k, gn = n0 + nq;
        const float* src = Bb + (int64_t)gk * p.ldb + gn;
        if (MODE == kLoadFast) {
          r[u] = ks_in_bounds(p, 1, src, 16) ? __ldg(reinterpret_cast<const float4*>(src)) : float4{};
          continue;
        }
        if (MODE == kLoadKTail) {
          r[u] = (gk < K && ks_in_bounds(p, 1, src, 16)) ? __ldg(reinterpret_cast<const float4*>(src)) : float4{};
          continue;
        }
        if (gk < K) load_vec_global<4>(v, src, p.N - gn, p.vecB, p, 1);
      } else {  // stored N x K: chunk along k
        const int n = c / (BK / 4), kq = (c % (BK / 4)) * 4;
        const int gn = n0 + n, gk = k0 + kq;
        const float* src = Bb + (int64_t)gn * p.ldb + gk;
        if (MODE == kLoadFast) {
          r[u] = ks_in_bounds(p, 1, src, 16) ? __ldg(reinterpret_cast<const float4*>(src)) : float4{};
          continue;
        }
        if (MODE == kLoadKTail || gn < p.N) load_vec_global<4>(v, src, K - gk, MODE == kLoadKTail || p.vecB, p, 1);
      }
    }
    r[u] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

template <class Cfg>
__device__ __forceinline__ void store_slice_b(const float4 (&r)[Cfg::RB], const GemmArgs& p, float* Bs, int tid) {
  constexpr int BK = Cfg::BK, BN = Cfg::BN, L = Cfg::LDS_B;
#pragma unroll
  for (int u = 0; u < Cfg::RB; ++u) {
    const int c = tid + u * Cfg::T;
    if (c < Cfg::CHB) {
      if (!p.transB) {
        const int k = c / (BN / 4), nq = (c % (BN / 4)) * 4;
        *reinterpret_cast<float4*>(Bs + k * L + Cfg::swz_b(nq, k)) = r[u];
      } else {
        const int n = c / (BK / 4), kq = (c % (BK / 4)) * 4;
        const int pn = Cfg::swz_b(n, kq);
        Bs[(kq + 0) * L + pn] = r[u].x;
        Bs[(kq + 1) * L + pn] = r[u].y;
        Bs[(kq + 2) * L + pn] = r[u].z;
        Bs[(kq + 3) * L + pn] = r[u].w;
      }
    }
  }
}

// The staged K loop: each BK slice of op(A) and op(B) is loaded into registers
// while the previous one (in the other half of the shared-memory ring) is
// consumed, then stored transposed to [k][m] / [k][n].  INTERIOR: every row and
// column of the tile is in range and 16-byte loads are legal, so full slices are
// read without checks and only a slice past K checks k.  Otherwise every load
// checks every bound.
template <class Cfg, bool INTERIOR>
__device__ __forceinline__ void staged_loop(const GemmArgs& p, const float* Ab, const float* Bb, int m0, int n0,
                                            int K, int tid, int tx, int ty, AccTile<Cfg::TM, Cfg::TN>& acc) {
  constexpr int TM = Cfg::TM, TN = Cfg::TN, BK = Cfg::BK, CM = Cfg::CM, CN = Cfg::CN;
  constexpr int PART = INTERIOR ? kLoadKTail : kLoadGeneral;
  extern __shared__ __align__(16) float smem[];
  float4 ra[Cfg::RA], rb[Cfg::RB];
  const int nk = (K + BK - 1) / BK;
  if (INTERIOR && BK <= K) {
    load_slice_a<Cfg, kLoadFast>(ra, p, Ab, m0, 0, K, tid);
    load_slice_b<Cfg, kLoadFast>(rb, p, Bb, n0, 0, K, tid);
  } else {
    load_slice_a<Cfg, PART>(ra, p, Ab, m0, 0, K, tid);
    load_slice_b<Cfg, PART>(rb, p, Bb, n0, 0, K, tid);
  }
  store_slice_a<Cfg>(ra, p, smem, tid);
  store_slice_b<Cfg>(rb, p, smem + BK * Cfg::LDS_A, tid);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const float* As = smem + (kt & 1) * Cfg::STAGE_FLOATS;
    const float* Bs = As + BK * Cfg::LDS_A;
    const bool more = kt + 1 < nk;
    if (more) {
      const int kn = (kt + 1) * BK;
      if (INTERIOR && kn + BK <= K) {
        load_slice_a<Cfg, kLoadFast>(ra, p, Ab, m0, kn, K, tid);
        load_slice_b<Cfg, kLoadFast>(rb, p, Bb, n0, kn, K, tid);
      } else {
        load_slice_a<Cfg, PART>(ra, p, Ab, m0, kn, K, tid);
        load_slice_b<Cfg, PART>(rb, p, Bb, n0, kn, K, tid);
      }
    }
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float a[TM], bv[TN];
#pragma unroll
      for (int ic = 0; ic < TM / CM; ++ic)
        load_vec_smem<CM>(a + ic * CM, As + k * Cfg::LDS_A + Cfg::swz_a(ic * (Cfg::WY * CM) + ty * CM, k));
#pragma unroll
      for (int jc = 0; jc < TN / CN; ++jc)
        load_vec_smem<CN>(bv + jc * CN, Bs + k * Cfg::LDS_B + Cfg::swz_b(jc * (Cfg::WX * CN) + tx * CN, k));
      acc.fma(a, bv);
    }
    if (more) {
      float* An = smem + ((kt + 1) & 1) * Cfg::STAGE_FLOATS;
      store_slice_a<Cfg>(ra, p, An, tid);
      store_slice_b<Cfg>(rb, p, An + BK * Cfg::LDS_A, tid);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- kernel
template <class Cfg, bool SPLIT>
__global__ void __launch_bounds__(Cfg::T) simt_gemm_kernel(const GemmArgs p) {
  constexpr int TM = Cfg::TM, TN = Cfg::TN, BK = Cfg::BK, CM = Cfg::CM, CN = Cfg::CN;
  pdl_wait();
  pdl_launch_dependents();
  const int tid = threadIdx.x;
  int tx, ty;
  thread_coords<Cfg>(tid, tx, ty);
  const int m0 = blockIdx.x * Cfg::BM, n0 = blockIdx.y * Cfg::BN;
  // SPLIT instances: blockIdx.z enumerates (batch entry, K split) pairs, split
  // s covers k in [s * kchunk, min(K, (s + 1) * kchunk)) and writes its own
  // partial tile (C then points at the split workspace, one M x ldc slab per z).
  // Otherwise blockIdx.z is the batch entry and the CTA covers all of K.
  const int z = blockIdx.z;
  int b = z, K = p.K;
  int64_t offA = 0, offB = 0;
  if constexpr (SPLIT) {
    b = z / p.splits;
    const int kbeg = (z - b * p.splits) * p.kchunk;
    K = min(p.K - kbeg, p.kchunk);
    offA = p.transA ? (int64_t)kbeg * p.lda : kbeg;
    offB = p.transB ? kbeg : (int64_t)kbeg * p.ldb;
  }
  const float* Ab = static_cast<const float*>(p.A) + (int64_t)b * p.strideA + offA;
  const float* Bb = static_cast<const float*>(p.B) + (int64_t)b * p.strideB + offB;
  float* Cb = p.C + (int64_t)z * p.strideC;

  AccTile<TM, TN> acc;
  acc.zero();

  const int nk = (K + BK - 1) / BK;
  if constexpr (Cfg::STAGED) {
    // Interior tiles with 16-byte-loadable operands run a loop whose loads check
    // nothing but the K tail; edge tiles and unaligned operands run the general one.
    const bool interior = (m0 + Cfg::BM <= p.M) && (n0 + Cfg::BN <= p.N) && p.vecA && p.vecB;
    if (interior) staged_loop<Cfg, true>(p, Ab, Bb, m0, n0, K, tid, tx, ty, acc);
    else staged_loop<Cfg, false>(p, Ab, Bb, m0, n0, K, tid, tx, ty, acc);
  } else {
    // Direct: every thread reads its own rows of op(A) and columns of op(B).
    for (int kt = 0; kt < nk; ++kt) {
#pragma unroll
      for (int kq = 0; kq < BK; kq += 4) {
        const int gk = kt * BK + kq;
        if (gk >= K) break;
        const int klim = K - gk;
        float a[TM][4], bv[4][TN];
        if (!p.transA) {
#pragma unroll
          for (int i = 0; i < TM; ++i) {
            const int gm = m0 + Cfg::row(i, ty);
            if (gm < p.M) {
              load_vec_global<4>(a[i], Ab + (int64_t)gm * p.lda + gk, klim, p.vecA, p, 0);
            } else {
              a[i][0] = a[i][1] = a[i][2] = a[i][3] = 0.f;
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int ic = 0; ic < TM / CM; ++ic) {
              const int r0 = ic * (Cfg::WY * CM) + ty * CM;
              float t[CM];
              if (k < klim) {
                load_vec_global<CM>(t, Ab + (int64_t)(gk + k) * p.lda + m0 + r0, p.M - m0 - r0, p.vecA, p, 0);
              } else {
#pragma unroll
                for (int q = 0; q < CM; ++q) t[q] = 0.f;
              }
#pragma unroll
              for (int q = 0; q < CM; ++q) a[ic * CM + q][k] = t[q];
            }
        }
        if (!p.transB) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int jc = 0; jc < TN / CN; ++jc) {
              const int c0 = jc * (Cfg::WX * CN) + tx * CN;
              float t[CN];
              if (k < klim) {
                load_vec_global<CN>(t, Bb + (int64_t)(gk + k) * p.ldb + n0 + c0, p.N - n0 - c0, p.vecB, p, 1);
              } else {
#pragma unroll
                for (int q = 0; q < CN; ++q) t[q] = 0.f;
              }
#pragma unroll
              for (int q = 0; q < CN; ++q) bv[k][jc * CN + q] = t[q];
            }
        } else {
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            const int gn = n0 + Cfg::col(j, tx);
            float t[4] = {0.f, 0.f, 0.f, 0.f};
            if (gn < p.N) load_vec_global<4>(t, Bb + (int64_t)gn * p.ldb + gk, klim, p.vecB, p, 1);
#pragma unroll
            for (int k = 0; k < 4; ++k) bv[k][j] = t[k];
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          float ak[TM];
#pragma unroll
          for (int i = 0; i < TM; ++i) ak[i] = a[i][k];
          acc.fma(ak, bv[k]);
        }
      }
    }
  }
  float out[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) out[i][j] = acc.get(i, j);
  int etx, ety;  // recomputed rather than kept live through the K loop
  thread_coords<Cfg>(threadIdx.x, etx, ety);
  epilogue<Cfg>(p, Cb, m0, n0, etx, ety, out);
}

template <int ID, bool SPLIT = false>
cudaError_t launch_simt(const GemmArgs& a, cudaStream_t s) {
  constexpr SimtParams P = simt_params(ID);
  using Cfg = SimtCfg<P.tm, P.tn, P.wx, P.wy, P.bk, P.staged != 0>;
  auto kern = simt_gemm_kernel<Cfg, SPLIT>;
  if constexpr (Cfg::SMEM_BYTES > 48 * 1024) {
    static unsigned long long done_mask = 0;  // devices whose attribute is set
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(__atomic_load_n(&done_mask, __ATOMIC_ACQUIRE) & bit)) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM_BYTES);
      if (e != cudaSuccess) return e;
      __atomic_fetch_or(&done_mask, bit, __ATOMIC_ACQ_REL);
    }
  }
  dim3 grid((a.M + Cfg::BM - 1) / Cfg::BM, (a.N + Cfg::BN - 1) / Cfg::BN, SPLIT ? a.batch * a.splits : a.batch);
  return launch_pdl(kern, grid, dim3(Cfg::T), Cfg::SMEM_BYTES, s, nullptr, 0, a);
}

// Resident CTAs per SM of the split instance of config ID on the current device (0 on error).
template <int ID>
int occupancy_simt() {
  constexpr SimtParams P = simt_params(ID);
  using Cfg = SimtCfg<P.tm, P.tn, P.wx, P.wy, P.bk, P.staged != 0>;
  auto kern = simt_gemm_kernel<Cfg, true>;
  if constexpr (Cfg::SMEM_BYTES > 48 * 1024) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM_BYTES) != cudaSuccess)
      return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, Cfg::T, Cfg::SMEM_BYTES) != cudaSuccess) return 0;
  return n;
}

}  // namespace ks
