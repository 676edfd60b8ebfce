// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/kselect.h"

namespace ks {

// ------------------------------------------------------------------ programmatic dependent launch
// The GEMM path's kernels are launched with programmatic stream serialisation:
// a kernel may be scheduled while the previous kernel in the stream drains
// (its launch and prologue overlap that tail), so it passes pdl_wait() before
// its first access to global memory, which returns once the previous grid has
// completed and its writes are visible (immediately when launched without the
// attribute).  pdl_launch_dependents() lets the next kernel be scheduled as
// soon as every CTA of this grid has run it; the next kernel still waits for
// this grid to complete before touching memory.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch `kern` with programmatic stream serialisation (plus `extra`
// attributes); only for kernels that call pdl_wait() before touching memory.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       const cudaLaunchAttribute* extra, int n_extra, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[4];
  int n = 0;
  for (int i = 0; i < n_extra && n < 3; ++i) attr[n++] = extra[i];
  attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[n].val.programmaticStreamSerializationAllowed = 1;
  ++n;
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = n;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// ------------------------------------------------------------------ FP32 SIMT config space
// id = ((((tm_i * 4 + tn_i) * 6 + wg_i) * 3 + bk_i) * 2 + staged); see kselect.h.
constexpr int kSimtConfigs = 576;
struct SimtParams {
  int tm, tn, wx, wy, bk, staged;
};

// Work-group shapes (WX, WY): 8x8, 16x16, 32x8, 8x32, 16x8, 8x16.
constexpr int simt_wg_x(int w) { return w == 0 ? 8 : w == 1 ? 16 : w == 2 ? 32 : w == 3 ? 8 : w == 4 ? 16 : 8; }
constexpr int simt_wg_y(int w) { return w == 0 ? 8 : w == 1 ? 16 : w == 2 ? 8 : w == 3 ? 32 : w == 4 ? 8 : 16; }

constexpr SimtParams simt_params(int id) {
  return SimtParams{1 << ((id / 144) % 4), 1 << ((id / 36) % 4), simt_wg_x((id / 6) % 6),
                    simt_wg_y((id / 6) % 6), 8 << ((id / 2) % 3), id % 2};
}

// Arguments of one (batched) GEMM launch, already validated by the host.
struct GemmArgs {
  int M, N, K, batch;
  int transA, transB;  // 1 = 'T'
  float alpha, beta;
  const void* A;
  int64_t lda, strideA;
  const void* B;
  int64_t ldb, strideB;
  float* C;
  int64_t ldc, strideC;
  int vecA, vecB, vecC;  // 16-byte vector access is legal on this operand
  // K split (SIMT family): blockIdx.z = batch entry * splits + split; split s
  // covers k in [s * kchunk, min(K, (s + 1) * kchunk)) and C/ldc/strideC then
  // describe the partial-sum workspace (one M x ldc slab per z).
  int splits = 1, kchunk = 0;
#ifdef KS_DEBUG_BOUNDS
  // Debug build: the bytes each operand may touch from its base (A, B, C), and
  // the device counter of accesses found outside them (each one is skipped).
  const char* lo[3] = {nullptr, nullptr, nullptr};
  int64_t ext[3] = {0, 0, 0};
  int* err = nullptr;
#endif
};

// True when [ptr, ptr + bytes) lies inside operand `op`'s extent; always true
// outside the debug build (the check compiles away).
__device__ __forceinline__ bool ks_in_bounds(const GemmArgs& p, int op, const void* ptr, int bytes) {
#ifdef KS_DEBUG_BOUNDS
  const char* c = static_cast<const char*>(ptr);
  if (c < p.lo[op] || c + bytes > p.lo[op] + p.ext[op]) {
    atomicAdd(p.err, 1);
    return false;
  }
#endif
  return true;
}

using LaunchFn = cudaError_t (*)(const GemmArgs&, cudaStream_t);
using OccFn = int (*)();  // resident CTAs per SM on the current device, 0 on error

// Per-shard registration of the SIMT instantiations (simt_shard.cu compiled N times).
constexpr int kSimtShards = 12;

// ------------------------------------------------------------------ split-K kind
// Config id kSplitBase + b runs SIMT config b with its K range divided among
// CTAs when the output tiles alone would leave most of the GPU's resident-CTA
// slots empty; the partial tiles are summed by a second kernel.  The kind
// covers the staged configs with BK in {16, 32} (192 ids).
constexpr int kSplitBase = 2000;
constexpr int kSplitConfigs = 192;
constexpr bool split_eligible(int base) {
  return base >= 0 && base < kSimtConfigs && (base % 2) == 1 && ((base / 2) % 3) != 0;
}

// Tensor-core families (tc_gemm.cu).
constexpr int kTcBase = 1000;
constexpr int kTcConfigsPerFamily = 18;
bool tc_config_valid(int id);
gemm_status_t tc_launch(int id, const GemmArgs& a, cudaStream_t s);
gemm_status_t tc_params(int id, int32_t out[8]);

void set_last_cuda_error(cudaError_t e);

}  // namespace ks

// The library handle: an immutable deployment plus a per-device cache of the
// MLP parameters (filled on first use by select_kernels_batched).
// The selector's feature row of one size (Section 5.1 reads the sizes; the
// fifth feature is the number of outputs, M * N * batch).
inline void selector_features(int64_t M, int64_t N, int64_t K, int64_t batch, double f[GEMM_TREE_FEATURES]) {
  f[0] = (double)M;
  f[1] = (double)N;
  f[2] = (double)K;
  f[3] = (double)batch;
  f[4] = (double)M * (double)N * (double)batch;
}

struct kselect_library {
  int precision;
  std::vector<int32_t> ids;
  std::vector<gemm_tree_node_t> nodes;
  std::vector<int32_t> roots;  // forest: one root per tree; empty: one tree rooted at 0
  std::vector<float> mlp;  // empty when absent
  std::vector<std::array<int64_t, 4>> known;  // sorted benchmarked sizes
  std::vector<int32_t> known_ids;
  std::mutex dev_mu;
  float* dev_mlp[64] = {nullptr};
  // gemm_grouped's workspace per device (descriptors, pre-pass jobs and
  // scratch); buffers it outgrew stay allocated until the handle is destroyed,
  // because graphs captured earlier still name them.
  char* dev_ws[64] = {nullptr};
  int64_t dev_ws_bytes[64] = {0};
  std::vector<char*> retired_ws;
  ~kselect_library() {
    for (float* p : dev_mlp)
      if (p) cudaFree(p);
    for (char* p : dev_ws)
      if (p) cudaFree(p);
    for (char* p : retired_ws) cudaFree(p);
  }
};
