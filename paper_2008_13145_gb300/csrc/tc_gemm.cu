// Tensor-core GEMM families on sm_103a: TF32, BF16 and split-BF16 x3, for a
// single batched GEMM and for an uneven group of GEMMs in one launch.
//
// The kernel (tc_kernel.cuh) consumes two K-contiguous operands.  op(A) = A
// with A stored M x K is used in place, op(B) = B^T with B stored N x K too;
// other layouts, and operands whose rows are not 16-byte aligned, are first
// rewritten K-contiguous by a tiled transpose pre-pass into scratch.  The x3
// family splits each FP32 value x into hi = bf16(x) and lo = bf16(x - hi) in
// the same pre-pass and lays K out as three segments, A' = [hi | hi | lo] and
// B' = [hi | lo | hi], so one BF16 GEMM over K' = 3 K accumulates
// hi*hi + hi*lo + lo*hi in FP32.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <cstring>
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
  int pair;    // 1: clusters of two CTAs sharing the B slice by multicast
};

bool decode(int id, TcConfig* c) {
  if (id < kTcBase) return false;
  const int fam = (id - kTcBase) / 100, idx = (id - kTcBase) % 100;
  if (fam < 0 || fam > 2 || idx >= kTcConfigsPerFamily) return false;
  c->family = fam + 1;
  c->bn = kTcBn[idx / 6];
  c->stages = kTcStages[(idx / 2) % 3];
  c->pair = idx % 2;
  return true;
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
// (inner, rows) = (K, R); MN-major ones (R, K).
bool make_map(CUtensorMap* m, const void* base, bool bf16, int64_t K, int64_t rows, int64_t ld, int64_t batch,
              int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int64_t elem = bf16 ? 2 : 4;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * elem), (cuuint64_t)(ld * elem * rows)};
  cuuint32_t box[3] = {(cuuint32_t)(128 / elem), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ---------------------------------------------------------------- device status word (sticky)
int* status_word() {
  static int* words[64] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> g(mu);
  if (!words[dev]) {
    int* w = nullptr;
    if (cudaMalloc(&w, sizeof(int)) != cudaSuccess) return nullptr;
    if (cudaMemset(w, 0, sizeof(int)) != cudaSuccess) return nullptr;
    words[dev] = w;
  }
  return words[dev];
}

// ---------------------------------------------------------------- K-contiguous pre-pass
// One rewrite job: out[b][r][seg * Kp + k] for r < R, k < Kp (zero for k >= K)
// from the logical R x K operand whose element (r, k) of batch entry b sits at
// in[b * in_stride + r * rs + k * ks].  Copy (nseg 1, same type) or x3 split
// (FP32 in, BF16 out, nseg 2: segment 0 holds hi, segment 1 lo, as bit s of
// `pattern` set = segment s holds lo).
struct PrepJob {
  const void* in;
  int64_t in_stride, rs, ks;
  void* out;
  int64_t ld_out;
  int R, K, Kp, nseg, pattern;
  int tiles_k, tiles_r, block_start;  // 64 x 64 tiles; first block of this job (grouped form)
  int vec2;  // element pairs along the source's contiguous dimension may be read as one access
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

template <typename TIn, typename TOut, bool SPLIT>
__device__ __forceinline__ void prep_tile(const PrepJob& j, int b, int tr, int tk) {
  __shared__ float tile[64][65];
  pdl_wait();
  pdl_launch_dependents();
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
      const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
      const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
      const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
      __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(dst) + (int64_t)r * j.ld_out + k;
      for (int sg = 0; sg < j.nseg; ++sg) {
        const bool lo = (j.pattern >> sg) & 1;
        __nv_bfloat16* os = o + (int64_t)sg * j.Kp;
        if (two) *reinterpret_cast<__nv_bfloat162*>(os) = __halves2bfloat162(lo ? l0 : h0, lo ? l1 : h1);
        else os[0] = lo ? l0 : h0;
      }
    }
  }
}

// Batched form: grid (tiles_k, tiles_r, batch).
template <typename TIn, typename TOut, bool SPLIT>
__global__ void prep_kernel(const PrepJob j) {
  prep_tile<TIn, TOut, SPLIT>(j, blockIdx.z, blockIdx.y, blockIdx.x);
}

// Grouped form: one block per (job, tile); jobs sorted by block_start.
template <typename TIn, typename TOut, bool SPLIT>
__global__ void prep_group_kernel(const PrepJob* jobs, int n_jobs) {
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
  // The job table is written once when the plan is made, so reading it before
  // the programmatic wait in prep_tile is safe.
  if (family == GEMM_PREC_F32X3)
    return launch_pdl(prep_group_kernel<float, __nv_bfloat16, true>, dim3(blocks), block, 0, s, nullptr, 0, jobs, n_jobs);
  if (family == GEMM_PREC_BF16)
    return launch_pdl(prep_group_kernel<__nv_bfloat16, __nv_bfloat16, false>, dim3(blocks), block, 0, s, nullptr, 0,
                      jobs, n_jobs);
  return launch_pdl(prep_group_kernel<float, float, false>, dim3(blocks), block, 0, s, nullptr, 0, jobs, n_jobs);
}

// ---------------------------------------------------------------- main kernel launch
// Persistent grid: one CTA (or CTA pair) per resident slot, at most one per tile unit.
template <int BN, int STAGES, bool TF32, bool GROUPED, bool PAIR>
cudaError_t launch_kernel(const CUtensorMap& ma, const CUtensorMap& mb, const tc::TcArgs& a, const tc::GroupArgs& g,
                          cudaStream_t s) {
  using Cfg = tc::TcCfg<BN, STAGES, TF32>;
  auto kern = tc::tc_gemm_kernel<BN, STAGES, TF32, GROUPED, PAIR>;
  static unsigned long long done_mask = 0;
  static int slots_cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.blockDim = dim3(tc::kThreads, 1, 1);
  cfg.dynamicSmemBytes = Cfg::SMEM_BYTES;
  cfg.stream = s;
  if (PAIR) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  if (!(__atomic_load_n(&done_mask, __ATOMIC_ACQUIRE) & bit)) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    // Resident CTAs per SM from the kernel's own resources: shared memory
    // (plus what the system reserves per CTA), registers and TMEM columns.
    // The runtime's occupancy query reports one CTA per SM for these kernels
    // whatever their size, while the SM runs as many as these resources allow.
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    int smem_sm = 0, sms = 0, reserved = 0, regs_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    const int regs = (fa.numRegs + 7) / 8 * 8;
    int occ = std::min(smem_sm / (Cfg::SMEM_BYTES + (int)fa.sharedSizeBytes + reserved), regs_sm / (regs * tc::kThreads));
    occ = std::max(1, std::min(occ, 512 / Cfg::TMEM_COLS));  // every resident CTA must fit in TMEM
    int slots = occ * sms;
    if (PAIR) {
      // The cluster query places one pair per two SMs; scale it by the CTAs per SM.
      int clusters = 0;
      cfg.gridDim = dim3(2 * sms, 1, 1);
      e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
      if (e != cudaSuccess) return e;
      slots = std::max(1, std::min(clusters * occ, slots / 2));  // in pairs
    }
    slots_cache[dev & 63] = slots;
    __atomic_fetch_or(&done_mask, bit, __ATOMIC_ACQ_REL);
  }
  const int units = std::min(a.num_tiles, slots_cache[dev & 63]);
  return launch_pdl(kern, dim3((unsigned)(PAIR ? 2 * units : units), 1, 1), cfg.blockDim, cfg.dynamicSmemBytes, s,
                    cfg.attrs, (int)cfg.numAttrs, ma, mb, a, g);
}

using TcLaunch = cudaError_t (*)(const CUtensorMap&, const CUtensorMap&, const tc::TcArgs&, const tc::GroupArgs&,
                                 cudaStream_t);

template <bool TF32, bool GROUPED, bool PAIR>
TcLaunch pick(int bn, int stages) {
#define KS_TC_CASE(B, S) \
  if (bn == B && stages == S) return &launch_kernel<B, S, TF32, GROUPED, PAIR>;
  KS_TC_CASE(64, 2) KS_TC_CASE(64, 3) KS_TC_CASE(64, 4)
  KS_TC_CASE(128, 2) KS_TC_CASE(128, 3) KS_TC_CASE(128, 4)
  KS_TC_CASE(256, 2) KS_TC_CASE(256, 3) KS_TC_CASE(256, 4)
#undef KS_TC_CASE
  return nullptr;
}

TcLaunch pick_launch(const TcConfig& c, bool grouped) {
  const bool tf32 = c.family == GEMM_PREC_TF32;
  if (c.pair) {
    if (grouped) return tf32 ? pick<true, true, true>(c.bn, c.stages) : pick<false, true, true>(c.bn, c.stages);
    return tf32 ? pick<true, false, true>(c.bn, c.stages) : pick<false, false, true>(c.bn, c.stages);
  }
  if (grouped) return tf32 ? pick<true, true, false>(c.bn, c.stages) : pick<false, true, false>(c.bn, c.stages);
  return tf32 ? pick<true, false, false>(c.bn, c.stages) : pick<false, false, false>(c.bn, c.stages);
}

// Row-tile units: 128-row tiles, or pairs of them.
int row_units(int64_t M, int pair) {
  const int t = (int)((M + tc::kBM - 1) / tc::kBM);
  return pair ? (t + 1) / 2 : t;
}

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
// the extent along R that one CTA loads per slice (128 for A, BN or BN / 2 for B).
OperandPlan plan_operand(const TcConfig& c, const void* ptr, int64_t ld, int64_t stride, bool kcontig, int R, int K,
                         int batch, int pattern, int mn_ext) {
  const bool x3 = c.family == GEMM_PREC_F32X3;
  const int64_t in_elem = c.family == GEMM_PREC_BF16 ? 2 : 4;
  const int64_t op_elem = c.family == GEMM_PREC_TF32 ? 4 : 2;
  OperandPlan o;
  // Read in place only when K-contiguous, 16-byte aligned and batch-packed (the
  // tensor map's third dimension steps R x ld); otherwise the pre-pass packs it.
  o.direct = !x3 && kcontig && ((uintptr_t)ptr % 16 == 0) && ((ld * in_elem) % 16 == 0) &&
             (batch == 1 || stride == (int64_t)R * ld);
  // A BF16 operand stored K x R (R contiguous) is read in place as MN-major
  // tiles of whole 64-wide boxes when it is 16-byte aligned and batch-packed
  // (K x ld per entry).
  o.mn = !o.direct && c.family == GEMM_PREC_BF16 && !kcontig && mn_ext % tc::kMnBox == 0 &&
         ((uintptr_t)ptr % 16 == 0) && ((ld * in_elem) % 16 == 0) && (batch == 1 || stride == (int64_t)K * ld);
  if (o.mn) o.direct = true;
  const int nseg = x3 ? 2 : 1;
  const int64_t Kp = x3 ? round_up(K, 64) : round_up(K, 16 / op_elem);
  o.ld = o.direct ? ld : nseg * Kp;
  o.bytes = o.direct ? 0 : (int64_t)batch * R * o.ld * op_elem;
  // Element pairs along the contiguous dimension are read as one access when
  // every pair starts on a multiple of two elements: base, row and batch
  // strides all even multiples of the element size.
  const int64_t pair_bytes = 2 * in_elem;
  const int vec2 = ((uintptr_t)ptr % pair_bytes == 0) && (ld % 2 == 0) && (stride % 2 == 0);
  o.job = PrepJob{ptr, stride, kcontig ? ld : 1, kcontig ? 1 : ld, nullptr, o.ld, R, K, (int)Kp, nseg, pattern,
                  (int)((Kp + 63) / 64), (R + 63) / 64, 0, vec2};
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
  int32_t v[8] = {c.family, 128, c.bn, bk, c.stages, c.pair, 0, 0};
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
  const int b_ext = c.pair ? c.bn / 2 : c.bn;
  OperandPlan pa = plan_operand(c, g.A, g.lda, g.strideA, !g.transA, g.M, g.K, g.batch, /*hi,lo*/ 0b10, tc::kBM);
  OperandPlan pb = plan_operand(c, g.B, g.ldb, g.strideB, g.transB != 0, g.N, g.K, g.batch, /*hi,lo*/ 0b10, b_ext);
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
  // x3: the K' loop covers 3 segments of round_up(K, 64); the operands hold 2.
  const bool x3 = c.family == GEMM_PREC_F32X3;
  const int64_t Kop = x3 ? 3 * round_up(g.K, 64) : g.K;
  const int64_t Kmap = x3 ? 2 * round_up(g.K, 64) : g.K;
  CUtensorMap ma, mb;
  const int bk = op_bf16 ? 64 : 32;
  const bool map_ok = st == GEMM_OK &&
                      (pa.mn ? make_map(&ma, Aop, op_bf16, g.M, Kmap, pa.ld, g.batch, bk)
                             : make_map(&ma, Aop, op_bf16, Kmap, g.M, pa.ld, g.batch, tc::kBM)) &&
                      (pb.mn ? make_map(&mb, Bop, op_bf16, g.N, Kmap, pb.ld, g.batch, bk)
                             : make_map(&mb, Bop, op_bf16, Kmap, g.N, pb.ld, g.batch, b_ext));
  if (st == GEMM_OK && !map_ok) st = GEMM_ERR_MISALIGNED;
  if (st == GEMM_OK) {
    tc::TcArgs a;
    a.M = g.M; a.N = g.N; a.K = (int)Kop; a.batch = g.batch;
    a.tiles_m = row_units(g.M, c.pair);
    a.tiles_n = (g.N + c.bn - 1) / c.bn;
    a.num_tiles = a.tiles_m * a.tiles_n * g.batch;
    a.k_blocks = (int)((Kop + (op_bf16 ? 63 : 31)) / (op_bf16 ? 64 : 32));
    // Grouped raster: 8 tile rows (units) per group bound the operand slices the
    // SMs' tiles in flight read at once (8 A + ~10 B slices for 152 CTAs).
    a.raster = 2;
    a.group_m = std::max(1, std::min(a.tiles_m, kRasterGroup));
    a.alpha = g.alpha; a.beta = g.beta;
    a.C = g.C; a.ldc = g.ldc; a.strideC = g.strideC; a.vecC = g.vecC;
    a.a_mn = pa.mn; a.b_mn = pb.mn;
    a.seg_blocks = x3 ? (int)(round_up(g.K, 64) / 64) : 0;
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

// ------------------------------------------------------------------ grouped plans
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
  const bool op_bf16 = c.family != GEMM_PREC_TF32;
  const int64_t op_elem = op_bf16 ? 2 : 4;
  std::vector<tc::GroupDesc> descs(count);
  std::vector<PrepJob> jobs;
  std::vector<OperandPlan> pa(count), pb(count);
  int64_t scratch_bytes = 0, tiles = 0;
  std::vector<int64_t> offA(count, -1), offB(count, -1);
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
    pa[i] = plan_operand(c, q.A, q.lda, 0, !ta, (int)q.M, (int)q.K, 1, /*hi,lo*/ 0b10, tc::kBM);
    pb[i] = plan_operand(c, q.B, q.ldb, 0, tb != 0, (int)q.N, (int)q.K, 1, /*hi,lo*/ 0b10, c.pair ? c.bn / 2 : c.bn);
    if (!pa[i].direct) { offA[i] = scratch_bytes; scratch_bytes += round_up(pa[i].bytes, 256); }
    if (!pb[i].direct) { offB[i] = scratch_bytes; scratch_bytes += round_up(pb[i].bytes, 256); }
    const int tm = row_units(q.M, c.pair), tn = (int)((q.N + c.bn - 1) / c.bn);
    tiles += (int64_t)tm * tn;
    if (tiles >= (1ll << 31)) return GEMM_ERR_UNSUPPORTED;
  }
  kselect_grouped_plan* p = new (std::nothrow) kselect_grouped_plan();
  if (!p) return GEMM_ERR_UNSUPPORTED;
  p->cfg = c;
  p->count = count;
  cudaGetDevice(&p->device);
  cudaError_t e = cudaSuccess;
  if (scratch_bytes > 0) e = cudaMalloc(reinterpret_cast<void**>(&p->scratch), scratch_bytes);
  if (e != cudaSuccess) { plan_free(p); return fail(e); }
  // Tiles are dealt to the persistent CTAs by static striding over the global
  // tile index, so the problems are laid out by K-steps per tile, longest
  // first: each CTA then takes one tile per round of a longest-first list,
  // which balances uneven groups (results do not depend on the order).
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  const int64_t kmul = c.family == GEMM_PREC_F32X3 ? 3 : 1;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const int64_t kx = kmul * (c.family == GEMM_PREC_F32X3 ? round_up(probs[x].K, 64) : probs[x].K);
    const int64_t ky = kmul * (c.family == GEMM_PREC_F32X3 ? round_up(probs[y].K, 64) : probs[y].K);
    return kx > ky;
  });
  int tile_start = 0, blocks = 0;
  for (int r = 0; r < count; ++r) {
    const int i = order[r];
    const gemm_problem_t& q = probs[i];
    const void* Aop = pa[i].direct ? q.A : p->scratch + offA[i];
    const void* Bop = pb[i].direct ? q.B : p->scratch + offB[i];
    if (!pa[i].direct) {
      pa[i].job.out = const_cast<void*>(Aop);
      pa[i].job.block_start = blocks;
      blocks += pa[i].job.tiles_k * pa[i].job.tiles_r;
      jobs.push_back(pa[i].job);
    }
    if (!pb[i].direct) {
      pb[i].job.out = const_cast<void*>(Bop);
      pb[i].job.block_start = blocks;
      blocks += pb[i].job.tiles_k * pb[i].job.tiles_r;
      jobs.push_back(pb[i].job);
    }
    const bool x3 = c.family == GEMM_PREC_F32X3;
    const int64_t Kop = x3 ? 3 * round_up(q.K, 64) : q.K;  // K' loop; the operands hold 2 segments
    const int64_t Kmap = x3 ? 2 * round_up(q.K, 64) : q.K;
    tc::GroupDesc& d = descs[r];
    std::memset(&d, 0, sizeof(d));
    const int64_t Mr = q.M > 0 ? q.M : 1, Nr = q.N > 0 ? q.N : 1;
    const int bk = op_bf16 ? 64 : 32;
    const bool ok_a = pa[i].mn ? make_map(&d.tmA, Aop, op_bf16, Mr, Kmap, pa[i].ld, 1, bk)
                               : make_map(&d.tmA, Aop, op_bf16, Kmap, Mr, pa[i].ld, 1, tc::kBM);
    const bool ok_b = pb[i].mn ? make_map(&d.tmB, Bop, op_bf16, Nr, Kmap, pb[i].ld, 1, bk)
                               : make_map(&d.tmB, Bop, op_bf16, Kmap, Nr, pb[i].ld, 1, c.pair ? c.bn / 2 : c.bn);
    if (!ok_a || !ok_b) {
      plan_free(p);
      return GEMM_ERR_MISALIGNED;
    }
    d.C = q.C;
    d.ldc = q.ldc;
    d.M = (int)q.M;
    d.N = (int)q.N;
    d.k_blocks = (int)((Kop * op_elem + 127) / 128);
    d.tiles_m = row_units(q.M, c.pair);
    d.tiles_n = (int)((q.N + c.bn - 1) / c.bn);
    d.tile_start = tile_start;
    d.vecC = ((uintptr_t)q.C % 16 == 0) && (q.ldc % 4 == 0);
    d.a_mn = pa[i].mn;
    d.b_mn = pb[i].mn;
    d.seg_blocks = x3 ? (int)(round_up(q.K, 64) / 64) : 0;
    d.alpha = q.alpha;
    d.beta = q.beta;
    tile_start += d.tiles_m * d.tiles_n;
  }
  p->total_tiles = tile_start;
  p->n_jobs = (int)jobs.size();
  p->prep_blocks = blocks;
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
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* status = status_word();
  if (!status) return fail(cudaGetLastError());
  cudaError_t e = launch_prep_group(p->cfg.family, p->jobs, p->n_jobs, p->prep_blocks, s);
  if (e != cudaSuccess) return fail(e);
  TcLaunch fn = pick_launch(p->cfg, true);
  if (!fn) return GEMM_ERR_NO_KERNEL;
  tc::TcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.num_tiles = p->total_tiles;
  a.raster = 0;
  a.status = status;
  tc::GroupArgs g{p->descs, p->count};
  CUtensorMap dummy;
  std::memset(&dummy, 0, sizeof(dummy));
  e = fn(dummy, dummy, a, g, s);
  return e == cudaSuccess ? GEMM_OK : fail(e);
}

void gemm_grouped_plan_destroy(gemm_grouped_plan_t p) { plan_free(p); }

gemm_status_t gemm_grouped(int32_t id, int32_t count, const gemm_problem_t* probs, void* stream) {
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
