// Tensor-core GEMM families on sm_103a: TF32, BF16 and split-BF16 x3, for a
// single batched GEMM and for an uneven group of GEMMs in one launch.
//
// The kernel (tc_kernel.cuh) reads each operand in place when its rows are
// 16-byte aligned and batch-packed: K-contiguous (A stored M x K, B stored
// N x K) as K-major tiles, MN-contiguous (A stored K x M, B stored K x N) as
// MN-major tiles.  Other operands, and every x3 operand, are first rewritten
// K-contiguous by a tiled transpose pre-pass into scratch.  The x3
// family splits each FP32 value x into hi = bf16(x) and lo = bf16(x - hi) in
// the same pre-pass and stores [hi | lo] per row; the kernel's K' = 3 K loop
// reads the segment pairs (hi, hi), (hi, lo), (lo, hi), so one BF16 GEMM
// accumulates hi*hi + hi*lo + lo*hi in FP32 (for K < 64, three parts and six
// products: see split_plan).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <numeric>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "tc_kernel.cuh"

namespace ks {
namespace {
constexpr int kRasterGroup = 8;

constexpr int kTcBn[3] = {64, 128, 256};
constexpr int kTcStages[3] = {2, 3, 4};

struct TcConfig {
  int family;  // GEMM_PREC_TF32, GEMM_PREC_BF16, GEMM_PREC_F32X3
  int bn, stages;
};

// Index idx of a family is (BN slot * 3 + stage slot) * 2 + p; the slots with
// p = 1 are reserved (no kernel), so a family has 9 valid configurations.
bool decode(int id, TcConfig* c) {
  if (id < kTcBase) return false;
  const int fam = (id - kTcBase) / 100, idx = (id - kTcBase) % 100;
  if (fam < 0 || fam > 2 || idx >= kTcConfigsPerFamily || idx % 2 != 0) return false;
  c->family = fam + 1;
  c->bn = kTcBn[idx / 6];
  c->stages = kTcStages[(idx / 2) % 3];
  return true;
}

// ---------------------------------------------------------------- split-BF16 products (F32X3 family)
// Each FP32 operand x is split into BF16 parts x = p0 + p1 (+ p2) + r, each
// part the rounded remainder of the previous ones, and the K' loop runs one
// K-segment per product of parts.  BF16 keeps 8 significant bits, so with two
// parts the three products p0q0 + p0q1 + p1q0 drop terms of up to 3 * 2^-16 of
// |xy| per product; summed over K products of uniform data these errors
// average out below 1e-5 of sum |xy| once K reaches a few tens, but not for
// K of a few.  Below kSplit6MaxK the family therefore uses three parts and
// the six products whose part indexes sum to at most 2, which drop terms
// below about 4 * 2^-24 of |xy|: the FP32 level at every K.  Small-K products
// are bound by memory and launch latency, so the extra products cost little.
constexpr int64_t kSplit6MaxK = 64;
constexpr int64_t kSplitSeg = 64;  // K elements per segment are padded to a whole 128-byte slice

struct SplitPlan {
  int nseg;     // parts per operand (segments stored)
  int nprod;    // products (segments of the K' loop)
  int seg_map;  // product g: A part at bits [2g, 2g + 2), B part at bits [16 + 2g, 16 + 2g + 2)
};

SplitPlan split_plan(int64_t K) {
  static constexpr int a3[3] = {0, 0, 1}, b3[3] = {0, 1, 0};
  static constexpr int a6[6] = {0, 0, 1, 0, 1, 2}, b6[6] = {0, 1, 0, 2, 1, 0};
  const bool six = K < kSplit6MaxK;
  SplitPlan p{six ? 3 : 2, six ? 6 : 3, 0};
  for (int g = 0; g < p.nprod; ++g)
    p.seg_map |= ((six ? a6[g] : a3[g]) << (2 * g)) | ((six ? b6[g] : b3[g]) << (16 + 2 * g));
  return p;
}

// ---------------------------------------------------------------- driver entry point for TMA descriptors
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 3-D map over a (batch, rows, inner) operand whose `inner` dimension is
// contiguous; box = (128-byte inner slice) x box_rows.  K-major operands pass
// (inner, rows) = (K, R); MN-major ones (R, K), and an MN-major FP32 operand
// (read as TF32) is swizzled in 32-byte pieces (atom32), the layout the MMA
// reads 32-bit MN-major operands in.
bool make_map(CUtensorMap* m, const void* base, bool bf16, int64_t K, int64_t rows, int64_t ld, int64_t batch,
              int box_rows, bool atom32 = false) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int64_t elem = bf16 ? 2 : 4;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * elem), (cuuint64_t)(ld * elem * rows)};
  cuuint32_t box[3] = {(cuuint32_t)(128 / elem), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  atom32 ? CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B : CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ---------------------------------------------------------------- device status word (sticky)
// One int per device, made by the device's first tensor-core call; with
// create = false a device that has none yet gets nullptr (nothing allocated).
int* status_word_of(bool create) {
  static int* words[64] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> g(mu);
  if (!words[dev] && create) {
    int* w = nullptr;
    if (cudaMalloc(&w, sizeof(int)) != cudaSuccess) return nullptr;
    if (cudaMemset(w, 0, sizeof(int)) != cudaSuccess) return nullptr;
    words[dev] = w;
  }
  return words[dev];
}

int* status_word() { return status_word_of(true); }
int* status_word_if_ready() { return status_word_of(false); }

// ---------------------------------------------------------------- K-contiguous pre-pass
// One rewrite job: out[b][r][seg * Kp + k] for r < R, k < Kp (zero for k >= K)
// from the logical R x K operand whose element (r, k) of batch entry b sits at
// in[b * in_stride + r * rs + k * ks]; with mn_out (a split of an FP32 operand
// stored MN-contiguous) the parts are written MN-major instead,
// out[b][seg * Kp + k][r], without a transpose.  Copy (nseg 1, same type) or BF16
// split (FP32 in, BF16 out, nseg 2 or 3): segment 0 holds p0 = bf16(x) and
// segment s the rounded remainder p_s = bf16(x - p0 - ... - p_{s-1}); every
// remainder is exact in FP32.
struct PrepJob {
  const void* in;
  int64_t in_stride, rs, ks;
  void* out;
  int64_t ld_out;
  int R, K, Kp, nseg;
  int tiles_k, tiles_r, block_start;  // 64 x 64 tiles; first block of this job (grouped form)
  int vec2;  // element pairs along the source's contiguous dimension may be read as one access
  int vec4;  // FP32 source, every 4-element group along its contiguous dimension 16-byte aligned (direct split)
  int mn_out;  // write the parts MN-major (vec4 jobs of an MN-contiguous source only)
};

template <typename T>
__device__ __forceinline__ float to_f32(T v) {
  if constexpr (sizeof(T) == 2) return __bfloat162float(v);
  else return (float)v;
}

// One 64 x 64 tile of a job.  A warp row reads 64 consecutive elements along
// the source's contiguous dimension (two per lane, as one access when the job
// allows), the tile turns in shared memory, and a warp row writes 64
// consecutive K positions of one output row (two per lane).
constexpr int kPrepWarps = 8;  // warps per pre-pass block; each takes 64 / kPrepWarps tile rows

// Split of one 64 x 64 tile of an FP32 source whose contiguous dimension is
// 16-byte aligned, in the source's own orientation: each thread reads 4
// consecutive elements along the contiguous dimension as one 16-byte access
// and writes 4 BF16 of every part as one 8-byte store, without staging through
// shared memory (a warp covers two lines of the tile).  K-contiguous source:
// out row r holds the parts side by side along K.  MN-contiguous source
// (mn_out): out row (seg * Kp + k) holds part seg of column k, so the parts are
// stacked along K and the GEMM reads them MN-major.
__device__ __forceinline__ void split_tile_direct(const PrepJob& j, int b, int tr, int tk) {
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const float* src = static_cast<const float*>(j.in) + (int64_t)b * j.in_stride;
  const int64_t out_stride = j.mn_out ? (int64_t)j.nseg * j.Kp * j.ld_out : (int64_t)j.R * j.ld_out;
  __nv_bfloat16* dst = static_cast<__nv_bfloat16*>(j.out) + (int64_t)b * out_stride;
#pragma unroll
  for (int q = 0; q < 64 * 16 / (32 * kPrepWarps); ++q) {
    const int idx = q * 32 * kPrepWarps + tid;
    // (r, k) of the first of this thread's 4 elements; the 4 run along the contiguous dimension
    const int r = j.mn_out ? tr * 64 + (idx % 16) * 4 : tr * 64 + idx / 16;
    const int k = j.mn_out ? tk * 64 + idx / 16 : tk * 64 + (idx % 16) * 4;
    if (r >= j.R || k >= j.Kp) continue;
    const float* p = src + (int64_t)r * j.rs + (int64_t)k * j.ks;  // the step along the 4 is 1
    const int lim = j.mn_out ? (k < j.K ? j.R - r : 0) : j.K - k;   // how many of the 4 exist in the source
    float v[4];
    if (lim >= 4) {
      const float4 w = *reinterpret_cast<const float4*>(p);
      v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = (e < lim) ? p[e] : 0.f;
    }
    // ld_out is a multiple of 8 (MN-major) or of 64 (K-major), and Kp of 64: the stores are 8-byte aligned
    __nv_bfloat16* o = j.mn_out ? dst + (int64_t)k * j.ld_out + r : dst + (int64_t)r * j.ld_out + k;
    const int64_t seg_step = j.mn_out ? (int64_t)j.Kp * j.ld_out : (int64_t)j.Kp;
    for (int sg = 0; sg < j.nseg; ++sg) {
      __nv_bfloat16 part[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        part[e] = __float2bfloat16_rn(v[e]);
        v[e] -= __bfloat162float(part[e]);
      }
      const __nv_bfloat162 p01 = __halves2bfloat162(part[0], part[1]), p23 = __halves2bfloat162(part[2], part[3]);
      uint2 w;
      std::memcpy(&w.x, &p01, 4);
      std::memcpy(&w.y, &p23, 4);
      *reinterpret_cast<uint2*>(o + (int64_t)sg * seg_step) = w;
    }
  }
}

template <typename TIn, typename TOut, bool SPLIT>
__device__ __forceinline__ void prep_tile(const PrepJob& j, int b, int tr, int tk) {
  __shared__ float tile[64][65];
  pdl_wait();
  pdl_launch_dependents();
  if constexpr (SPLIT && sizeof(TIn) == 4) {
    if (j.vec4) {  // the same for every thread of the block
      split_tile_direct(j, b, tr, tk);
      return;
    }
  }
  const int r0 = tr * 64, k0 = tk * 64, lane = threadIdx.x;
  const TIn* src = static_cast<const TIn*>(j.in) + (int64_t)b * j.in_stride;
  const bool k_fast = (j.ks == 1);
#pragma unroll
  for (int it = 0; it < 64 / kPrepWarps; ++it) {
    const int i = threadIdx.y + it * kPrepWarps;
    int r, k;  // first element of this lane's pair; the second is the next along the contiguous dimension
    if (k_fast) { r = r0 + i; k = k0 + 2 * lane; } else { k = k0 + i; r = r0 + 2 * lane; }
    const bool in0 = r < j.R && k < j.K;
    const bool in1 = k_fast ? (r < j.R && k + 1 < j.K) : (r + 1 < j.R && k < j.K);
    const TIn* p = src + (int64_t)r * j.rs + (int64_t)k * j.ks;
    float v0 = 0.f, v1 = 0.f;
    if (j.vec2 && in1) {
      if constexpr (sizeof(TIn) == 2) {
        const __nv_bfloat162 w = *reinterpret_cast<const __nv_bfloat162*>(p);
        v0 = __low2float(w);
        v1 = __high2float(w);
      } else {
        const float2 w = *reinterpret_cast<const float2*>(p);
        v0 = w.x;
        v1 = w.y;
      }
    } else {
      if (in0) v0 = to_f32(p[0]);
      if (in1) v1 = to_f32(p[1]);
    }
    if (k_fast) { tile[i][2 * lane] = v0; tile[i][2 * lane + 1] = v1; }
    else { tile[2 * lane][i] = v0; tile[2 * lane + 1][i] = v1; }
  }
  __syncthreads();
  TOut* dst = static_cast<TOut*>(j.out) + (int64_t)b * j.R * j.ld_out;
#pragma unroll
  for (int it = 0; it < 64 / kPrepWarps; ++it) {
    const int i = threadIdx.y + it * kPrepWarps;
    const int r = r0 + i, k = k0 + 2 * lane;
    if (r >= j.R || k >= j.Kp) continue;
    const float x0 = tile[i][2 * lane], x1 = tile[i][2 * lane + 1];
    const bool two = k + 1 < j.Kp;  // Kp and ld_out are even, so a pair is 2-element aligned
    if constexpr (!SPLIT) {
      TOut* o = dst + (int64_t)r * j.ld_out + k;
      if constexpr (sizeof(TOut) == 2) {
        if (two) *reinterpret_cast<__nv_bfloat162*>(o) = __floats2bfloat162_rn(x0, x1);
        else o[0] = __float2bfloat16_rn(x0);
      } else {
        if (two) *reinterpret_cast<float2*>(o) = make_float2(x0, x1);
        else o[0] = x0;
      }
    } else {
      float r0 = x0, r1 = x1;  // remainders still to be represented
      __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(dst) + (int64_t)r * j.ld_out + k;
      for (int sg = 0; sg < j.nseg; ++sg) {
        const __nv_bfloat16 p0 = __float2bfloat16_rn(r0), p1 = __float2bfloat16_rn(r1);
        r0 -= __bfloat162float(p0);
        r1 -= __bfloat162float(p1);
        __nv_bfloat16* os = o + (int64_t)sg * j.Kp;
        if (two) *reinterpret_cast<__nv_bfloat162*>(os) = __halves2bfloat162(p0, p1);
        else os[0] = p0;
      }
    }
  }
}

// Batched form: grid (tiles_k, tiles_r, batch).
template <typename TIn, typename TOut, bool SPLIT>
__global__ void prep_kernel(const PrepJob j) {
  prep_tile<TIn, TOut, SPLIT>(j, blockIdx.z, blockIdx.y, blockIdx.x);
}

// Grouped form: one block per (job, tile); jobs sorted by block_start.  The
// job table may have been written by the kernel just before (gemm_grouped
// uploads it), so the programmatic wait comes before reading it.
template <typename TIn, typename TOut, bool SPLIT>
__global__ void prep_group_kernel(const PrepJob* jobs, int n_jobs) {
  pdl_wait();
  const int blk = blockIdx.x;
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].block_start <= blk) lo = mid; else hi = mid - 1;
  }
  const PrepJob j = jobs[lo];
  const int t = blk - j.block_start;
  prep_tile<TIn, TOut, SPLIT>(j, 0, t / j.tiles_k, t % j.tiles_k);
}

cudaError_t launch_prep(int family, const PrepJob& j, int batch, cudaStream_t s) {
  dim3 block(32, kPrepWarps), grid((unsigned)j.tiles_k, (unsigned)j.tiles_r, (unsigned)batch);
  if (family == GEMM_PREC_F32X3) return launch_pdl(prep_kernel<float, __nv_bfloat16, true>, grid, block, 0, s, nullptr, 0, j);
  if (family == GEMM_PREC_BF16)
    return launch_pdl(prep_kernel<__nv_bfloat16, __nv_bfloat16, false>, grid, block, 0, s, nullptr, 0, j);
  return launch_pdl(prep_kernel<float, float, false>, grid, block, 0, s, nullptr, 0, j);
}

// Both operands of one GEMM in a single launch: blocks [0, na) rewrite A, the
// rest B (one launch less when neither operand can be read in place).
template <typename TIn, typename TOut, bool SPLIT>
__global__ void prep_pair_kernel(const PrepJob ja, const PrepJob jb) {
  const int na = ja.tiles_k * ja.tiles_r;
  const int t = (int)blockIdx.x;
  if (t < na) prep_tile<TIn, TOut, SPLIT>(ja, blockIdx.z, t / ja.tiles_k, t % ja.tiles_k);
  else prep_tile<TIn, TOut, SPLIT>(jb, blockIdx.z, (t - na) / jb.tiles_k, (t - na) % jb.tiles_k);
}

cudaError_t launch_prep_pair(int family, const PrepJob& ja, const PrepJob& jb, int batch, cudaStream_t s) {
  dim3 block(32, kPrepWarps), grid((unsigned)(ja.tiles_k * ja.tiles_r + jb.tiles_k * jb.tiles_r), 1, (unsigned)batch);
  if (family == GEMM_PREC_F32X3)
    return launch_pdl(prep_pair_kernel<float, __nv_bfloat16, true>, grid, block, 0, s, nullptr, 0, ja, jb);
  if (family == GEMM_PREC_BF16)
    return launch_pdl(prep_pair_kernel<__nv_bfloat16, __nv_bfloat16, false>, grid, block, 0, s, nullptr, 0, ja, jb);
  return launch_pdl(prep_pair_kernel<float, float, false>, grid, block, 0, s, nullptr, 0, ja, jb);
}

cudaError_t launch_prep_group(int family, const PrepJob* jobs, int n_jobs, int blocks, cudaStream_t s) {
  if (n_jobs == 0) return cudaSuccess;
  dim3 block(32, kPrepWarps);
  if (family == GEMM_PREC_F32X3)
    return launch_pdl(prep_group_kernel<float, __nv_bfloat16, true>, dim3(blocks), block, 0, s, nullptr, 0, jobs, n_jobs);
  if (family == GEMM_PREC_BF16)
    return launch_pdl(prep_group_kernel<__nv_bfloat16, __nv_bfloat16, false>, dim3(blocks), block, 0, s, nullptr, 0,
                      jobs, n_jobs);
  return launch_pdl(prep_group_kernel<float, float, false>, dim3(blocks), block, 0, s, nullptr, 0, jobs, n_jobs);
}

// ---------------------------------------------------------------- main kernel launch
// Persistent grid: one CTA per resident slot, at most one per tile.
template <int BN, int STAGES, bool TF32, bool GROUPED>
cudaError_t launch_kernel(const CUtensorMap& ma, const CUtensorMap& mb, const tc::TcArgs& a, const tc::GroupArgs& g,
                          cudaStream_t s) {
  using Cfg = tc::TcCfg<BN, STAGES, TF32>;
  auto kern = tc::tc_gemm_kernel<BN, STAGES, TF32, GROUPED>;
  static unsigned long long done_mask = 0;
  static int slots_cache[64] = {0};
  static int dyn_cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(__atomic_load_n(&done_mask, __ATOMIC_ACQUIRE) & bit)) {
    // Resident CTAs per SM from the kernel's own resources: shared memory
    // (plus what the system reserves per CTA), registers and TMEM columns.
    // The runtime's occupancy query reports one CTA per SM for these kernels
    // whatever their size, while the SM runs as many as these resources allow.
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    int smem_sm = 0, sms = 0, reserved = 0, regs_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    const int regs = (fa.numRegs + 7) / 8 * 8;
    const int per_cta = (int)fa.sharedSizeBytes + reserved;
    const int occ_smem = smem_sm / (Cfg::SMEM_BYTES + per_cta);
    int occ = std::min(occ_smem, regs_sm / (regs * tc::kThreads));
    occ = std::max(1, std::min(occ, 512 / Cfg::TMEM_COLS));  // every resident CTA must fit in TMEM
    // Where shared memory alone would let more CTAs onto an SM than TMEM or the
    // registers hold (BN 128 and BN 256 with two stages), ask for enough of it that
    // it cannot.  Otherwise the block scheduler may place an extra CTA on an SM
    // whose TMEM is taken: it waits in tcgen05.alloc until a persistent CTA there
    // has finished all its tiles, while the grid, sized for `occ` CTAs per SM,
    // leaves other SMs idle.  The padding is never touched.
    int dyn = Cfg::SMEM_BYTES;
    if (occ_smem > occ) dyn = std::max(dyn, (smem_sm / (occ + 1) - per_cta + 16 + 15) / 16 * 16);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
    dyn_cache[dev & 63] = dyn;
    slots_cache[dev & 63] = occ * sms;
    __atomic_fetch_or(&done_mask, bit, __ATOMIC_ACQ_REL);
  }
  const int ctas = std::min(a.num_tiles, slots_cache[dev & 63]);
  return launch_pdl(kern, dim3((unsigned)ctas, 1, 1), dim3(tc::kThreads, 1, 1), (size_t)dyn_cache[dev & 63], s,
                    nullptr, 0, ma, mb, a, g);
}

using TcLaunch = cudaError_t (*)(const CUtensorMap&, const CUtensorMap&, const tc::TcArgs&, const tc::GroupArgs&,
                                 cudaStream_t);

template <bool TF32, bool GROUPED>
TcLaunch pick(int bn, int stages) {
#define KS_TC_CASE(B, S) \
  if (bn == B && stages == S) return &launch_kernel<B, S, TF32, GROUPED>;
  KS_TC_CASE(64, 2) KS_TC_CASE(64, 3) KS_TC_CASE(64, 4)
  KS_TC_CASE(128, 2) KS_TC_CASE(128, 3) KS_TC_CASE(128, 4)
  KS_TC_CASE(256, 2) KS_TC_CASE(256, 3) KS_TC_CASE(256, 4)
#undef KS_TC_CASE
  return nullptr;
}

TcLaunch pick_launch(const TcConfig& c, bool grouped) {
  const bool tf32 = c.family == GEMM_PREC_TF32;
  if (grouped) return tf32 ? pick<true, true>(c.bn, c.stages) : pick<false, true>(c.bn, c.stages);
  return tf32 ? pick<true, false>(c.bn, c.stages) : pick<false, false>(c.bn, c.stages);
}

int row_tiles(int64_t M) { return (int)((M + tc::kBM - 1) / tc::kBM); }

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

gemm_status_t fail(cudaError_t e) {
  set_last_cuda_error(e);
  return GEMM_ERR_CUDA;
}

// How one operand reaches the kernel: in place, or through a rewrite job.
struct OperandPlan {
  bool direct;
  bool mn;         // read in place as MN-major tiles (BF16 stored MN-contiguous)
  int64_t ld;      // leading dimension the kernel reads
  int64_t bytes;   // scratch bytes (0 when direct)
  PrepJob job;     // filled when !direct (out set later)
};

// Operand of logical shape R x K (rows of op(A), or columns of op(B) = rows of
// B^T).  `kcontig` says whether it is stored R x K (K contiguous); `mn_ext` is
// the extent along R that one CTA loads per slice (128 for A, BN for B).
OperandPlan plan_operand(const TcConfig& c, const void* ptr, int64_t ld, int64_t stride, bool kcontig, int R, int K,
                         int batch, int mn_ext) {
  const bool x3 = c.family == GEMM_PREC_F32X3;
  const int64_t in_elem = c.family == GEMM_PREC_BF16 ? 2 : 4;
  const int64_t op_elem = c.family == GEMM_PREC_TF32 ? 4 : 2;
  OperandPlan o;
  // Read in place only when K-contiguous, 16-byte aligned and batch-packed (the
  // tensor map's third dimension steps R x ld); otherwise the pre-pass packs it.
  o.direct = !x3 && kcontig && ((uintptr_t)ptr % 16 == 0) && ((ld * in_elem) % 16 == 0) &&
             (batch == 1 || stride == (int64_t)R * ld);
  // A BF16 or TF32 operand stored K x R (R contiguous) is read in place as
  // MN-major tiles of whole 128-byte boxes (64 BF16 or 32 FP32 elements) when
  // it is 16-byte aligned and batch-packed (K x ld per entry).
  o.mn = !o.direct && !x3 && !kcontig && mn_ext % (128 / op_elem) == 0 &&
         ((uintptr_t)ptr % 16 == 0) && ((ld * in_elem) % 16 == 0) && (batch == 1 || stride == (int64_t)K * ld);
  if (o.mn) o.direct = true;
  // Every x3 operand is split by the pre-pass; an aligned one is split in its
  // own orientation (vec4), and one stored K x R is then read MN-major.
  const int vec4 = x3 && ((uintptr_t)ptr % 16 == 0) && (ld % 4 == 0) && (stride % 4 == 0);
  const bool x3_mn = x3 && !kcontig && vec4 && mn_ext % (128 / op_elem) == 0;
  if (x3_mn) o.mn = true;
  const int nseg = x3 ? split_plan(K).nseg : 1;
  const int64_t Kp = x3 ? round_up(K, kSplitSeg) : round_up(K, 16 / op_elem);
  // Scratch rows: K-major parts side by side (nseg * Kp per row), or MN-major
  // rows of R elements padded to 16 bytes (nseg * Kp rows per batch entry).
  o.ld = o.direct ? ld : x3_mn ? round_up(R, 8) : nseg * Kp;
  o.bytes = o.direct ? 0 : x3_mn ? (int64_t)batch * nseg * Kp * o.ld * op_elem : (int64_t)batch * R * o.ld * op_elem;
  // Element pairs along the contiguous dimension are read as one access when
  // every pair starts on a multiple of two elements: base, row and batch
  // strides all even multiples of the element size.
  const int64_t pair_bytes = 2 * in_elem;
  const int vec2 = ((uintptr_t)ptr % pair_bytes == 0) && (ld % 2 == 0) && (stride % 2 == 0);
  o.job = PrepJob{ptr, stride, kcontig ? ld : 1, kcontig ? 1 : ld, nullptr, o.ld, R, K, (int)Kp, nseg,
                  (int)((Kp + 63) / 64), (R + 63) / 64, 0, vec2, vec4, x3_mn ? 1 : 0};
  return o;
}

}  // namespace

bool tc_config_valid(int id) {
  TcConfig c;
  return decode(id, &c);
}

gemm_status_t tc_params(int id, int32_t out[8]) {
  TcConfig c;
  if (!decode(id, &c)) return GEMM_ERR_NO_KERNEL;
  const int bk = (c.family == GEMM_PREC_TF32) ? 32 : 64;
  int32_t v[8] = {c.family, 128, c.bn, bk, c.stages, 0, 0, 0};
  std::memcpy(out, v, sizeof(v));
  return GEMM_OK;
}

gemm_status_t tc_launch(int id, const GemmArgs& g, cudaStream_t s) {
  TcConfig c;
  if (!decode(id, &c)) return GEMM_ERR_NO_KERNEL;
  const bool op_bf16 = c.family != GEMM_PREC_TF32;
  TcLaunch fn = pick_launch(c, false);
  if (!fn) return GEMM_ERR_NO_KERNEL;
  if (!encode_fn()) return GEMM_ERR_UNSUPPORTED;
  int* status = status_word();
  if (!status) return fail(cudaGetLastError());

  // op(A) rows are M, stored M x K when transA = 0; op(B)^T rows are N, stored N x K when transB = 1.
  const int b_ext = c.bn;
  OperandPlan pa = plan_operand(c, g.A, g.lda, g.strideA, !g.transA, g.M, g.K, g.batch, tc::kBM);
  OperandPlan pb = plan_operand(c, g.B, g.ldb, g.strideB, g.transB != 0, g.N, g.K, g.batch, b_ext);
  char* scratch = nullptr;
  if (pa.bytes + pb.bytes > 0) {
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), pa.bytes + pb.bytes + 256, s);
    if (e != cudaSuccess) return fail(e);
  }
  const void* Aop = pa.direct ? g.A : scratch;
  const void* Bop = pb.direct ? g.B : scratch + round_up(pa.bytes, 256);
  cudaError_t e = cudaSuccess;
  pa.job.out = const_cast<void*>(Aop);
  pb.job.out = const_cast<void*>(Bop);
  if (!pa.direct && !pb.direct) {
    e = launch_prep_pair(c.family, pa.job, pb.job, g.batch, s);
  } else if (!pa.direct) {
    e = launch_prep(c.family, pa.job, g.batch, s);
  } else if (!pb.direct) {
    e = launch_prep(c.family, pb.job, g.batch, s);
  }
  gemm_status_t st = e == cudaSuccess ? GEMM_OK : fail(e);
  // Split products: the K' loop covers one segment of round_up(K, 64) per
  // product; the operands hold one segment per part.
  const bool x3 = c.family == GEMM_PREC_F32X3;
  const SplitPlan sp = split_plan(g.K);
  const int64_t Kop = x3 ? sp.nprod * round_up(g.K, kSplitSeg) : g.K;
  const int64_t Kmap = x3 ? sp.nseg * round_up(g.K, kSplitSeg) : g.K;
  CUtensorMap ma, mb;
  const int bk = op_bf16 ? 64 : 32;
  const bool map_ok = st == GEMM_OK &&
                      (pa.mn ? make_map(&ma, Aop, op_bf16, g.M, Kmap, pa.ld, g.batch, bk, !op_bf16)
                             : make_map(&ma, Aop, op_bf16, Kmap, g.M, pa.ld, g.batch, tc::kBM)) &&
                      (pb.mn ? make_map(&mb, Bop, op_bf16, g.N, Kmap, pb.ld, g.batch, bk, !op_bf16)
                             : make_map(&mb, Bop, op_bf16, Kmap, g.N, pb.ld, g.batch, b_ext));
  if (st == GEMM_OK && !map_ok) st = GEMM_ERR_MISALIGNED;
  if (st == GEMM_OK) {
    tc::TcArgs a;
    a.M = g.M; a.N = g.N; a.K = (int)Kop; a.batch = g.batch;
    a.tiles_m = row_tiles(g.M);
    a.tiles_n = (g.N + c.bn - 1) / c.bn;
    a.num_tiles = a.tiles_m * a.tiles_n * g.batch;
    a.k_blocks = (int)((Kop + (op_bf16 ? 63 : 31)) / (op_bf16 ? 64 : 32));
    // Grouped raster: 8 tile rows per group bound the operand slices the
    // SMs' tiles in flight read at once (8 A + ~10 B slices for 152 CTAs).
    a.raster = 2;
    a.group_m = std::max(1, std::min(a.tiles_m, kRasterGroup));
    a.alpha = g.alpha; a.beta = g.beta;
    a.C = g.C; a.ldc = g.ldc; a.strideC = g.strideC; a.vecC = g.vecC;
    a.a_mn = pa.mn; a.b_mn = pb.mn;
    a.seg_blocks = x3 ? (int)(round_up(g.K, kSplitSeg) / 64) : 0;
    a.seg_map = x3 ? sp.seg_map : 0;
    a.status = status;
    tc::GroupArgs none{nullptr, 0};
    e = fn(ma, mb, a, none, s);
    if (e != cudaSuccess) st = fail(e);
  }
  if (scratch) cudaFreeAsync(scratch, s);
  return st;
}

}  // namespace ks

namespace ks {
// One warp waits, with the kernels' bounded wait and the given limit, on an
// mbarrier that nothing ever arrives at: the wait gives up, records the
// "slice never landed" code in the status word and the kernel returns.
__global__ void wait_selftest_kernel(int* status, uint64_t limit_ns, int* waited) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
  }
  __syncthreads();
  const bool ok = tc::mbar_wait_for(&bar, 0, status, tc::kStatusTimeoutFull, limit_ns);
  if (threadIdx.x == 0) *waited = ok ? 1 : 0;
}
}  // namespace ks

// ------------------------------------------------------------------ grouped launches
// A group is laid out on the host (validation, per-operand plans, scratch
// offsets, problem order), then encoded into per-problem descriptors and
// pre-pass jobs once its scratch address is known.  A plan keeps these in
// device buffers of its own; gemm_grouped writes them into the handle's
// workspace with kernels that carry them as launch parameters, so that a
// CUDA graph captured around the call holds its own copy of them.
namespace ks {
namespace {

struct GroupBuild {
  TcConfig c;
  int count = 0, n_jobs = 0;
  std::vector<OperandPlan> pa, pb;
  std::vector<int64_t> offA, offB;
  std::vector<int> order;
  int64_t scratch_bytes = 0;
};

// K extent of the kernel's loop for one problem (split products: one segment per product).
int64_t k_loop(const TcConfig& c, int64_t K) {
  return c.family == GEMM_PREC_F32X3 ? split_plan(K).nprod * round_up(K, kSplitSeg) : K;
}

gemm_status_t group_layout(const TcConfig& c, int count, const gemm_problem_t* probs, GroupBuild* b) {
  if (count < 1 || !probs) return GEMM_ERR_INVALID_ARG;
  b->c = c;
  b->count = count;
  b->pa.resize(count);
  b->pb.resize(count);
  b->offA.assign(count, -1);
  b->offB.assign(count, -1);
  int64_t tiles = 0;
  for (int i = 0; i < count; ++i) {
    const gemm_problem_t& q = probs[i];
    int ta, tb;
    auto tr = [](char t, int* o) {
      if (t == 'N' || t == 'n') { *o = 0; return true; }
      if (t == 'T' || t == 't') { *o = 1; return true; }
      return false;
    };
    if (!tr(q.transA, &ta) || !tr(q.transB, &tb)) return GEMM_ERR_INVALID_ARG;
    if (q.M < 0 || q.N < 0 || q.K < 1 || q.M >= (1ll << 31) || q.N >= (1ll << 31) || q.K >= (1ll << 31))
      return GEMM_ERR_INVALID_ARG;
    if (!q.A || !q.B || !q.C || q.ldc < q.N) return GEMM_ERR_INVALID_ARG;
    if (q.lda < (ta ? q.M : q.K) || q.ldb < (tb ? q.K : q.N)) return GEMM_ERR_INVALID_ARG;
    b->pa[i] = plan_operand(c, q.A, q.lda, 0, !ta, (int)q.M, (int)q.K, 1, tc::kBM);
    b->pb[i] = plan_operand(c, q.B, q.ldb, 0, tb != 0, (int)q.N, (int)q.K, 1, c.bn);
    if (!b->pa[i].direct) { b->offA[i] = b->scratch_bytes; b->scratch_bytes += round_up(b->pa[i].bytes, 256); ++b->n_jobs; }
    if (!b->pb[i].direct) { b->offB[i] = b->scratch_bytes; b->scratch_bytes += round_up(b->pb[i].bytes, 256); ++b->n_jobs; }
    tiles += (int64_t)row_tiles(q.M) * ((q.N + c.bn - 1) / c.bn);
    if (tiles >= (1ll << 31)) return GEMM_ERR_UNSUPPORTED;
  }
  // Tiles are dealt to the persistent CTAs by static striding over the global
  // tile index, so the problems are laid out by K-steps per tile, longest
  // first: each CTA then takes one tile per round of a longest-first list,
  // which balances uneven groups (results do not depend on the order).
  b->order.resize(count);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int x, int y) { return k_loop(c, probs[x].K) > k_loop(c, probs[y].K); });
  return GEMM_OK;
}

// Descriptors and pre-pass jobs of a laid-out group whose scratch starts at
// `scratch`; *total_tiles and *prep_blocks receive the two launches' sizes.
gemm_status_t group_encode(const GroupBuild& b, const gemm_problem_t* probs, char* scratch,
                           std::vector<tc::GroupDesc>* descs, std::vector<PrepJob>* jobs, int* total_tiles,
                           int* prep_blocks) {
  const TcConfig& c = b.c;
  const bool op_bf16 = c.family != GEMM_PREC_TF32;
  const bool x3 = c.family == GEMM_PREC_F32X3;
  const int64_t op_elem = op_bf16 ? 2 : 4;
  const int bk = op_bf16 ? 64 : 32;
  descs->assign(b.count, tc::GroupDesc{});
  jobs->clear();
  int tile_start = 0, blocks = 0;
  for (int r = 0; r < b.count; ++r) {
    const int i = b.order[r];
    const gemm_problem_t& q = probs[i];
    const OperandPlan& pa = b.pa[i];
    const OperandPlan& pb = b.pb[i];
    const void* Aop = pa.direct ? q.A : scratch + b.offA[i];
    const void* Bop = pb.direct ? q.B : scratch + b.offB[i];
    if (!pa.direct) {
      PrepJob j = pa.job;
      j.out = const_cast<void*>(Aop);
      j.block_start = blocks;
      blocks += j.tiles_k * j.tiles_r;
      jobs->push_back(j);
    }
    if (!pb.direct) {
      PrepJob j = pb.job;
      j.out = const_cast<void*>(Bop);
      j.block_start = blocks;
      blocks += j.tiles_k * j.tiles_r;
      jobs->push_back(j);
    }
    const SplitPlan sp = split_plan(q.K);
    const int64_t Kmap = x3 ? sp.nseg * round_up(q.K, kSplitSeg) : q.K;  // the operands hold one segment per part
    tc::GroupDesc& d = (*descs)[r];
    std::memset(&d, 0, sizeof(d));
    const int64_t Mr = q.M > 0 ? q.M : 1, Nr = q.N > 0 ? q.N : 1;
    const bool ok_a = pa.mn ? make_map(&d.tmA, Aop, op_bf16, Mr, Kmap, pa.ld, 1, bk, !op_bf16)
                            : make_map(&d.tmA, Aop, op_bf16, Kmap, Mr, pa.ld, 1, tc::kBM);
    const bool ok_b = pb.mn ? make_map(&d.tmB, Bop, op_bf16, Nr, Kmap, pb.ld, 1, bk, !op_bf16)
                            : make_map(&d.tmB, Bop, op_bf16, Kmap, Nr, pb.ld, 1, c.bn);
    if (!ok_a || !ok_b) return GEMM_ERR_MISALIGNED;
    d.C = q.C;
    d.ldc = q.ldc;
    d.M = (int)q.M;
    d.N = (int)q.N;
    d.k_blocks = (int)((k_loop(c, q.K) * op_elem + 127) / 128);
    d.tiles_m = row_tiles(q.M);
    d.tiles_n = (int)((q.N + c.bn - 1) / c.bn);
    d.tile_start = tile_start;
    d.vecC = ((uintptr_t)q.C % 16 == 0) && (q.ldc % 4 == 0);
    d.a_mn = pa.mn;
    d.b_mn = pb.mn;
    d.seg_blocks = x3 ? (int)(round_up(q.K, kSplitSeg) / 64) : 0;
    d.seg_map = x3 ? sp.seg_map : 0;
    d.alpha = q.alpha;
    d.beta = q.beta;
    tile_start += d.tiles_m * d.tiles_n;
  }
  *total_tiles = tile_start;
  *prep_blocks = blocks;
  return GEMM_OK;
}

// The pre-pass (when any operand needs one) and the persistent grouped launch.
cudaError_t launch_group(const TcConfig& c, const tc::GroupDesc* descs_dev, int count, const PrepJob* jobs_dev,
                         int n_jobs, int prep_blocks, int total_tiles, int* status, cudaStream_t s) {
  cudaError_t e = launch_prep_group(c.family, jobs_dev, n_jobs, prep_blocks, s);
  if (e != cudaSuccess) return e;
  TcLaunch fn = pick_launch(c, true);
  if (!fn) return cudaErrorInvalidDeviceFunction;
  tc::TcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.num_tiles = total_tiles;
  a.raster = 0;
  a.status = status;
  tc::GroupArgs g{descs_dev, count};
  CUtensorMap dummy;
  std::memset(&dummy, 0, sizeof(dummy));
  return fn(dummy, dummy, a, g, s);
}

// Host bytes written to device memory by a kernel that receives them as its
// launch parameter (at most 32,764 bytes of parameters per launch).  Inside a
// stream capture the bytes become part of the graph.
constexpr int kUploadBytes = 32 * 1024 - 512;
struct UploadChunk {
  uint8_t* dst;  // 16-byte aligned
  int n;
  alignas(16) uint8_t data[kUploadBytes];
};

__global__ void upload_kernel(const __grid_constant__ UploadChunk c) {
  const int n16 = c.n / 16;
  for (int i = threadIdx.x; i < n16; i += blockDim.x)
    reinterpret_cast<uint4*>(c.dst)[i] = reinterpret_cast<const uint4*>(c.data)[i];
  for (int i = n16 * 16 + threadIdx.x; i < c.n; i += blockDim.x) c.dst[i] = c.data[i];
}

cudaError_t upload(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  std::unique_ptr<UploadChunk> ch(new (std::nothrow) UploadChunk);
  if (!ch) return cudaErrorMemoryAllocation;
  for (size_t off = 0; off < bytes; off += kUploadBytes) {
    ch->dst = static_cast<uint8_t*>(dst) + off;
    ch->n = (int)std::min<size_t>(kUploadBytes, bytes - off);
    std::memcpy(ch->data, static_cast<const uint8_t*>(src) + off, ch->n);
    upload_kernel<<<1, 256, 0, s>>>(*ch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Workspace layout of a laid-out group: [descriptors | jobs | scratch], each
// part 256-byte aligned from a 256-byte aligned base.
struct WsLayout {
  int64_t jobs_off, scratch_off, bytes;
};
WsLayout ws_layout(const GroupBuild& b) {
  WsLayout w;
  w.jobs_off = round_up((int64_t)sizeof(tc::GroupDesc) * b.count, 256);
  w.scratch_off = w.jobs_off + round_up((int64_t)sizeof(PrepJob) * b.n_jobs, 256);
  w.bytes = w.scratch_off + b.scratch_bytes;
  return w;
}

// Family a precision class runs grouped: its own, or split-BF16 x3 for the
// FP32 class (the tensor-core family with FP32-level accuracy).
int grouped_family(int32_t precision) {
  if (precision == GEMM_PREC_F32) return GEMM_PREC_F32X3;
  if (precision >= GEMM_PREC_TF32 && precision <= GEMM_PREC_F32X3) return precision;
  return -1;
}

// The group's config from the handle's group selector, checked against the family.
gemm_status_t grouped_config(gemm_handle_t h, int32_t count, const gemm_problem_t* probs, int32_t precision,
                             TcConfig* c) {
  if (!h || count < 1 || !probs) return GEMM_ERR_INVALID_ARG;
  const int fam = grouped_family(precision);
  if (fam < 0) return GEMM_ERR_INVALID_ARG;
  const int32_t id = gemm_grouped_select(h, count, probs);
  if (id < 0) return (gemm_status_t)id;
  if (!decode(id, c) || c->family != fam) return GEMM_ERR_NO_KERNEL;
  return GEMM_OK;
}

// Makes the handle's workspace on the current device at least `bytes` long.
// The buffer it replaces is kept (queued work and captured graphs may still
// use it) and freed with the handle.  Called with h->dev_mu held.
gemm_status_t ws_reserve(gemm_handle_t h, int dev, int64_t bytes) {
  if (h->dev_ws_bytes[dev] >= bytes) return GEMM_OK;
  char* p = nullptr;
  const int64_t grow = std::max<int64_t>(bytes, 1 << 20);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), grow);
  if (e != cudaSuccess) return fail(e);
  if (h->dev_ws[dev]) h->retired_ws.push_back(h->dev_ws[dev]);
  h->dev_ws[dev] = p;
  h->dev_ws_bytes[dev] = grow;
  return GEMM_OK;
}

}  // namespace
}  // namespace ks

struct kselect_grouped_plan {
  ks::TcConfig cfg;
  int count = 0, total_tiles = 0, n_jobs = 0, prep_blocks = 0;
  ks::tc::GroupDesc* descs = nullptr;  // device
  ks::PrepJob* jobs = nullptr;          // device
  char* scratch = nullptr;              // device
  int device = 0;
};

namespace {
void plan_free(kselect_grouped_plan* p) {
  if (!p) return;
  if (p->descs) cudaFree(p->descs);
  if (p->jobs) cudaFree(p->jobs);
  if (p->scratch) cudaFree(p->scratch);
  delete p;
}
}  // namespace

using namespace ks;

extern "C" {

gemm_status_t gemm_grouped_plan_create(int32_t id, int32_t count, const gemm_problem_t* probs, void* stream,
                                       gemm_grouped_plan_t* out) {
  if (!out) return GEMM_ERR_INVALID_ARG;
  *out = nullptr;
  TcConfig c;
  if (!decode(id, &c)) return GEMM_ERR_NO_KERNEL;
  if (count < 1 || !probs) return GEMM_ERR_INVALID_ARG;
  if (!encode_fn()) return GEMM_ERR_UNSUPPORTED;
  if (!status_word()) return fail(cudaGetLastError());  // made now, so that runs never allocate
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GroupBuild b;
  gemm_status_t st = group_layout(c, count, probs, &b);
  if (st != GEMM_OK) return st;
  kselect_grouped_plan* p = new (std::nothrow) kselect_grouped_plan();
  if (!p) return GEMM_ERR_UNSUPPORTED;
  p->cfg = c;
  p->count = count;
  cudaGetDevice(&p->device);
  cudaError_t e = cudaSuccess;
  if (b.scratch_bytes > 0) e = cudaMalloc(reinterpret_cast<void**>(&p->scratch), b.scratch_bytes);
  if (e != cudaSuccess) { plan_free(p); return fail(e); }
  std::vector<tc::GroupDesc> descs;
  std::vector<PrepJob> jobs;
  st = group_encode(b, probs, p->scratch, &descs, &jobs, &p->total_tiles, &p->prep_blocks);
  if (st != GEMM_OK) { plan_free(p); return st; }
  p->n_jobs = (int)jobs.size();
  e = cudaMalloc(reinterpret_cast<void**>(&p->descs), sizeof(tc::GroupDesc) * count);
  if (e == cudaSuccess && !jobs.empty()) e = cudaMalloc(reinterpret_cast<void**>(&p->jobs), sizeof(PrepJob) * jobs.size());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->descs, descs.data(), sizeof(tc::GroupDesc) * count, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !jobs.empty())
    e = cudaMemcpyAsync(p->jobs, jobs.data(), sizeof(PrepJob) * jobs.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { plan_free(p); return fail(e); }
  *out = p;
  return GEMM_OK;
}

gemm_status_t gemm_grouped_run(gemm_grouped_plan_t p, void* stream) {
  if (!p) return GEMM_ERR_INVALID_ARG;
  if (p->total_tiles == 0) return GEMM_OK;
  int* status = status_word();
  if (!status) return fail(cudaGetLastError());
  cudaError_t e = launch_group(p->cfg, p->descs, p->count, p->jobs, p->n_jobs, p->prep_blocks, p->total_tiles,
                               status, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GEMM_OK : fail(e);
}

void gemm_grouped_plan_destroy(gemm_grouped_plan_t p) { plan_free(p); }

gemm_status_t gemm_grouped_with_config(int32_t id, int32_t count, const gemm_problem_t* probs, void* stream) {
  gemm_grouped_plan_t p = nullptr;
  gemm_status_t st = gemm_grouped_plan_create(id, count, probs, stream, &p);
  if (st != GEMM_OK) return st;
  st = gemm_grouped_run(p, stream);
  // The plan's device buffers are released once the launch has finished.
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  plan_free(p);
  if (st == GEMM_OK && e != cudaSuccess) st = fail(e);
  return st;
}

gemm_status_t gemm_grouped_reserve(gemm_handle_t h, int32_t count, const gemm_problem_t* probs, int32_t precision) {
  TcConfig c;
  gemm_status_t st = grouped_config(h, count, probs, precision, &c);
  if (st != GEMM_OK) return st;
  GroupBuild b;
  if ((st = group_layout(c, count, probs, &b)) != GEMM_OK) return st;
  if (!encode_fn()) return GEMM_ERR_UNSUPPORTED;
  if (!status_word()) return fail(cudaGetLastError());
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return GEMM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> g(h->dev_mu);
  return ws_reserve(h, dev, ws_layout(b).bytes);
}

gemm_status_t gemm_grouped(gemm_handle_t h, int32_t count, const gemm_problem_t* probs, int32_t precision,
                           void* stream) {
  TcConfig c;
  gemm_status_t st = grouped_config(h, count, probs, precision, &c);
  if (st != GEMM_OK) return st;
  GroupBuild b;
  if ((st = group_layout(c, count, probs, &b)) != GEMM_OK) return st;
  if (!encode_fn()) return GEMM_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return fail(e);
  int* status = nullptr;
  if (cap == cudaStreamCaptureStatusNone) {
    status = status_word();  // may allocate on the device's first tensor-core call
    if (!status) return fail(cudaGetLastError());
  } else {
    status = status_word_if_ready();
    if (!status) return GEMM_ERR_UNSUPPORTED;  // first call on this device under capture
  }
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return GEMM_ERR_UNSUPPORTED;
  const WsLayout w = ws_layout(b);
  std::lock_guard<std::mutex> g(h->dev_mu);
  if (h->dev_ws_bytes[dev] < w.bytes) {
    if (cap != cudaStreamCaptureStatusNone) return GEMM_ERR_UNSUPPORTED;  // never allocate inside a capture
    if ((st = ws_reserve(h, dev, w.bytes)) != GEMM_OK) return st;
  }
  char* base = h->dev_ws[dev];
  std::vector<tc::GroupDesc> descs;
  std::vector<PrepJob> jobs;
  int total_tiles = 0, prep_blocks = 0;
  if ((st = group_encode(b, probs, base + w.scratch_off, &descs, &jobs, &total_tiles, &prep_blocks)) != GEMM_OK)
    return st;
  if (total_tiles == 0) return GEMM_OK;
  e = upload(base, descs.data(), sizeof(tc::GroupDesc) * descs.size(), s);
  if (e == cudaSuccess && !jobs.empty()) e = upload(base + w.jobs_off, jobs.data(), sizeof(PrepJob) * jobs.size(), s);
  if (e == cudaSuccess)
    e = launch_group(c, reinterpret_cast<const tc::GroupDesc*>(base), count,
                     reinterpret_cast<const PrepJob*>(base + w.jobs_off), (int)jobs.size(), prep_blocks, total_tiles,
                     status, s);
  return e == cudaSuccess ? GEMM_OK : fail(e);
}

gemm_status_t kselect_wait_selftest(int64_t limit_ns, int32_t* waited_out, void* stream) {
  if (!waited_out || limit_ns < 1 || limit_ns > (int64_t)ks::tc::kWaitLimitNs) return GEMM_ERR_INVALID_ARG;
  int* w = status_word();
  if (!w) return fail(cudaGetLastError());
  int* flag = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&flag), sizeof(int), s);
  if (e != cudaSuccess) return fail(e);
  ks::wait_selftest_kernel<<<1, 32, 0, s>>>(w, (uint64_t)limit_ns, flag);
  int v = -1;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(flag, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(e);
  *waited_out = v;
  return GEMM_OK;
}

gemm_status_t gemm_device_status(int32_t* out_status, int32_t clear) {
  if (!out_status) return GEMM_ERR_INVALID_ARG;
  int* w = status_word();
  if (!w) return fail(cudaGetLastError());
  int v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear) e = cudaMemset(w, 0, sizeof(int));
  if (e != cudaSuccess) return fail(e);
  *out_status = v;
  return v == 0 ? GEMM_OK : GEMM_ERR_TIMEOUT;
}

}  // extern "C"
