// Tensor-core GEMM families on sm_103a: TF32, BF16 and split-BF16 x3.
//
// The kernel (tc_kernel.cuh) consumes two K-contiguous operands.  op(A) = A
// with A stored M x K is used in place, op(B) = B^T with B stored N x K too;
// other layouts, and operands whose rows are not 16-byte aligned, are first
// rewritten K-contiguous by a tiled transpose pre-pass into stream-ordered
// scratch.  The x3 family splits each FP32 value x into hi = bf16(x) and
// lo = bf16(x - hi) in the same pre-pass and lays the K dimension out as three
// segments, A' = [hi | hi | lo] and B' = [hi | lo | hi], so one BF16 GEMM over
// K' = 3 K accumulates hi*hi + hi*lo + lo*hi in FP32.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "common.cuh"
#include "tc_kernel.cuh"

namespace ks {
namespace {

constexpr int kTcBn[3] = {64, 128, 256};
constexpr int kTcStages[3] = {2, 3, 4};

struct TcConfig {
  int family;  // GEMM_PREC_TF32, GEMM_PREC_BF16, GEMM_PREC_F32X3
  int bn, stages, raster;
};

bool decode(int id, TcConfig* c) {
  if (id < kTcBase) return false;
  const int fam = (id - kTcBase) / 100, idx = (id - kTcBase) % 100;
  if (fam < 0 || fam > 2 || idx >= kTcConfigsPerFamily) return false;
  c->family = fam + 1;
  c->bn = kTcBn[idx / 6];
  c->stages = kTcStages[(idx / 2) % 3];
  c->raster = idx % 2;
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

// 3-D map over a (batch, rows, K) K-contiguous operand; box = (128-byte K slice) x box_rows.
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
// out[b][r][seg * Kp + k] for r < R, k < Kp (zero for k >= K) from an input
// whose element (r, k) sits at in[b * in_stride + r * rs + k * ks].
// MODE 0: copy (same element type); MODE 1: x3 split of FP32 into BF16 with
// segment pattern `pattern` (bit s set = segment s holds lo, else hi).
template <typename TIn, typename TOut, int MODE>
__global__ void kmajor_kernel(const TIn* __restrict__ in, int64_t in_stride, int64_t rs, int64_t ks, int R, int K,
                              int Kp, int nseg, int pattern, TOut* __restrict__ out, int64_t ld_out) {
  __shared__ float tile[32][33];
  const int b = blockIdx.z;
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const TIn* src = in + (int64_t)b * in_stride;
  const bool k_fast = (ks == 1);
  // load 32 x 32 (coalesced along whichever index is contiguous in memory)
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    int r, k;
    if (k_fast) { r = r0 + i; k = k0 + threadIdx.x; } else { k = k0 + i; r = r0 + threadIdx.x; }
    float v = 0.f;
    if (r < R && k < K) {
      if constexpr (sizeof(TIn) == 2) v = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(src + r * rs + k * ks));
      else v = (float)src[r * rs + k * ks];
    }
    if (k_fast) tile[i][threadIdx.x] = v; else tile[threadIdx.x][i] = v;
  }
  __syncthreads();
  TOut* dst = out + (int64_t)b * R * ld_out;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, k = k0 + threadIdx.x;
    if (r >= R || k >= Kp) continue;
    const float x = tile[i][threadIdx.x];
    if constexpr (MODE == 0) {
      if constexpr (sizeof(TOut) == 2) {
        reinterpret_cast<__nv_bfloat16*>(dst)[(int64_t)r * ld_out + k] = __float2bfloat16_rn(x);
      } else {
        dst[(int64_t)r * ld_out + k] = x;
      }
    } else {
      const __nv_bfloat16 hi = __float2bfloat16_rn(x);
      const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
      __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(dst) + (int64_t)r * ld_out + k;
      for (int s = 0; s < nseg; ++s) o[(int64_t)s * Kp] = ((pattern >> s) & 1) ? lo : hi;
    }
  }
}

template <int BN, int STAGES, bool TF32>
cudaError_t launch_kernel(const CUtensorMap& ma, const CUtensorMap& mb, const tc::TcArgs& a, cudaStream_t s) {
  using Cfg = tc::TcCfg<BN, STAGES, TF32>;
  auto kern = tc::tc_gemm_kernel<BN, STAGES, TF32>;
  static unsigned long long done_mask = 0;
  static int occ_cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(__atomic_load_n(&done_mask, __ATOMIC_ACQUIRE) & bit)) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    int occ = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, tc::kThreads, Cfg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    occ = occ < 512 / Cfg::TMEM_COLS ? occ : 512 / Cfg::TMEM_COLS;  // every resident CTA must fit in TMEM
    occ_cache[dev & 63] = (occ < 1 ? 1 : occ) * sms;
    __atomic_fetch_or(&done_mask, bit, __ATOMIC_ACQ_REL);
  }
  const int slots = occ_cache[dev & 63];
  const int grid = a.num_tiles < slots ? a.num_tiles : slots;
  kern<<<grid, tc::kThreads, Cfg::SMEM_BYTES, s>>>(ma, mb, a);
  return cudaGetLastError();
}

using TcLaunch = cudaError_t (*)(const CUtensorMap&, const CUtensorMap&, const tc::TcArgs&, cudaStream_t);

template <bool TF32>
TcLaunch pick(int bn, int stages) {
#define KS_TC_CASE(B, S) \
  if (bn == B && stages == S) return &launch_kernel<B, S, TF32>;
  KS_TC_CASE(64, 2) KS_TC_CASE(64, 3) KS_TC_CASE(64, 4)
  KS_TC_CASE(128, 2) KS_TC_CASE(128, 3) KS_TC_CASE(128, 4)
  KS_TC_CASE(256, 2) KS_TC_CASE(256, 3) KS_TC_CASE(256, 4)
#undef KS_TC_CASE
  return nullptr;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

gemm_status_t fail(cudaError_t e) {
  set_last_cuda_error(e);
  return GEMM_ERR_CUDA;
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
  int32_t v[8] = {c.family, 128, c.bn, bk, c.stages, c.raster, 0, 0};
  std::memcpy(out, v, sizeof(v));
  return GEMM_OK;
}

gemm_status_t tc_launch(int id, const GemmArgs& g, cudaStream_t s) {
  TcConfig c;
  if (!decode(id, &c)) return GEMM_ERR_NO_KERNEL;
  const bool tf32 = (c.family == GEMM_PREC_TF32);
  const bool x3 = (c.family == GEMM_PREC_F32X3);
  const bool in_bf16 = (c.family == GEMM_PREC_BF16);
  const bool op_bf16 = !tf32;  // element type the tensor core reads
  const int64_t in_elem = in_bf16 ? 2 : 4, op_elem = op_bf16 ? 2 : 4;
  TcLaunch fn = tf32 ? pick<true>(c.bn, c.stages) : pick<false>(c.bn, c.stages);
  if (!fn) return GEMM_ERR_NO_KERNEL;
  if (!encode_fn()) return GEMM_ERR_UNSUPPORTED;
  int* status = status_word();
  if (!status) return fail(cudaGetLastError());

  // Operand layout: A as (batch, M, K) K-contiguous, B as (batch, N, K).
  const int per16 = (int)(16 / in_elem);
  const bool a_direct = !x3 && !g.transA && ((uintptr_t)g.A % 16 == 0) && (g.lda % per16 == 0);
  const bool b_direct = !x3 && g.transB && ((uintptr_t)g.B % 16 == 0) && (g.ldb % per16 == 0);
  const int nseg = x3 ? 3 : 1;
  const int64_t Kp = x3 ? round_up(g.K, 64) : round_up(g.K, 16 / op_elem);
  const int64_t ldA = a_direct ? g.lda : nseg * Kp, ldB = b_direct ? g.ldb : nseg * Kp;
  const int64_t bytesA = a_direct ? 0 : (int64_t)g.batch * g.M * ldA * op_elem;
  const int64_t bytesB = b_direct ? 0 : (int64_t)g.batch * g.N * ldB * op_elem;
  char* scratch = nullptr;
  if (bytesA + bytesB > 0) {
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), bytesA + bytesB + 256, s);
    if (e != cudaSuccess) return fail(e);
  }
  const void* Aop = a_direct ? g.A : scratch;
  const void* Bop = b_direct ? g.B : scratch + round_up(bytesA, 256);
  cudaError_t e = cudaSuccess;
  auto prep = [&](const void* in, int64_t in_stride, int trans, int64_t ld, int R, void* out, int64_t ld_out,
                  int pattern) {
    // element (r, k) of the logical R x K operand: stored R x K (trans 0) or K x R (trans 1)
    const int64_t rs = trans ? 1 : ld, kst = trans ? ld : 1;
    dim3 block(32, 8), grid((unsigned)((Kp + 31) / 32), (unsigned)((R + 31) / 32), (unsigned)g.batch);
    if (x3) {
      kmajor_kernel<float, __nv_bfloat16, 1><<<grid, block, 0, s>>>(
          static_cast<const float*>(in), in_stride, rs, kst, R, g.K, (int)Kp, nseg, pattern,
          static_cast<__nv_bfloat16*>(out), ld_out);
    } else if (in_bf16) {
      kmajor_kernel<__nv_bfloat16, __nv_bfloat16, 0><<<grid, block, 0, s>>>(
          static_cast<const __nv_bfloat16*>(in), in_stride, rs, kst, R, g.K, (int)Kp, 1, 0,
          static_cast<__nv_bfloat16*>(out), ld_out);
    } else {
      kmajor_kernel<float, float, 0><<<grid, block, 0, s>>>(static_cast<const float*>(in), in_stride, rs, kst, R,
                                                             g.K, (int)Kp, 1, 0, static_cast<float*>(out), ld_out);
    }
    return cudaGetLastError();
  };
  // op(A) rows are M: stored M x K when transA = 0.  op(B)^T rows are N: B is
  // stored N x K when transB = 1, i.e. "transposed" relative to (N, K) when 0.
  if (!a_direct) e = prep(g.A, g.strideA, g.transA, g.lda, g.M, const_cast<void*>(Aop), ldA, /*hi,hi,lo*/ 0b100);
  if (e == cudaSuccess && !b_direct)
    e = prep(g.B, g.strideB, g.transB ? 0 : 1, g.ldb, g.N, const_cast<void*>(Bop), ldB, /*hi,lo,hi*/ 0b010);
  gemm_status_t st = GEMM_OK;
  if (e != cudaSuccess) st = fail(e);
  const int64_t Kop = x3 ? 3 * Kp : g.K;
  CUtensorMap ma, mb;
  if (st == GEMM_OK) {
    if (!make_map(&ma, Aop, op_bf16, Kop, g.M, ldA, g.batch, tc::kBM) ||
        !make_map(&mb, Bop, op_bf16, Kop, g.N, ldB, g.batch, c.bn))
      st = GEMM_ERR_MISALIGNED;
  }
  if (st == GEMM_OK) {
    tc::TcArgs a;
    a.M = g.M; a.N = g.N; a.K = (int)Kop; a.batch = g.batch;
    a.tiles_m = (g.M + tc::kBM - 1) / tc::kBM;
    a.tiles_n = (g.N + c.bn - 1) / c.bn;
    a.num_tiles = a.tiles_m * a.tiles_n * g.batch;
    a.k_blocks = (int)((Kop + (op_bf16 ? 63 : 31)) / (op_bf16 ? 64 : 32));
    a.raster = c.raster;
    a.alpha = g.alpha; a.beta = g.beta;
    a.C = g.C; a.ldc = g.ldc; a.strideC = g.strideC; a.vecC = g.vecC;
    a.status = status;
    e = fn(ma, mb, a, s);
    if (e != cudaSuccess) st = fail(e);
  }
  if (scratch) cudaFreeAsync(scratch, s);
  return st;
}

}  // namespace ks

extern "C" gemm_status_t gemm_device_status(int32_t* out_status, int32_t clear) {
  if (!out_status) return GEMM_ERR_INVALID_ARG;
  int* w = ks::status_word();
  if (!w) return ks::fail(cudaGetLastError());
  int v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear) e = cudaMemset(w, 0, sizeof(int));
  if (e != cudaSuccess) return ks::fail(e);
  *out_status = v;
  return v == 0 ? GEMM_OK : GEMM_ERR_TIMEOUT;
}
