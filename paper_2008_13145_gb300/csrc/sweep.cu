// Benchmark every configuration on one set of sizes (Section 3.1).
//
// The paper times each (sizes, configuration) pair with warm-up launches and
// a timed run of back-to-back iterations lasting about a second.  A GB300
// sweep covers ~576k pairs, so the time budget is spent where it decides the
// result: pass 1 times one warm launch of every configuration; pass 2 re-times
// with a full back-to-back run only the configurations whose probe is within
// `refine_ratio` of the fastest probe.  The others keep their probe time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace ks {
gemm_status_t launch_by_id(int id, const GemmArgs& a, cudaStream_t s);
gemm_status_t make_launch_args(int id, char transA, char transB, int64_t M, int64_t N, int64_t K, float alpha,
                               const void* A, int64_t lda, const void* B, int64_t ldb, float beta, float* C,
                               int64_t ldc, int64_t batch, GemmArgs* a, bool* noop);
}  // namespace ks

using namespace ks;

static constexpr float kLongMs = 2.0f;

extern "C" gemm_status_t gemm_benchmark_configs(int32_t n_configs, const int32_t* config_ids, char transA,
                                                char transB, int64_t M, int64_t N, int64_t K, const void* A,
                                                int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc,
                                                int64_t batch, int32_t warmup, int32_t min_reps, int32_t max_reps,
                                                double min_total_ms, double refine_ratio, double* out_ms,
                                                int32_t* out_status, double* out_probe_ms, int32_t* out_reps,
                                                void* stream) {
  if (n_configs < 0 || (n_configs > 0 && (!config_ids || !out_ms || !out_status))) return GEMM_ERR_INVALID_ARG;
  if (warmup < 0 || min_reps < 1 || max_reps < min_reps || refine_ratio < 1.0) return GEMM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    set_last_cuda_error(cudaGetLastError());
    if (e0) cudaEventDestroy(e0);
    return GEMM_ERR_CUDA;
  }
  gemm_status_t ret = GEMM_OK;
  std::vector<GemmArgs> args(n_configs);
  double best = INFINITY;
  // Pass 1: warm-up launches and one timed probe launch per configuration.
  for (int c = 0; c < n_configs && ret == GEMM_OK; ++c) {
    out_ms[c] = 0.0;
    if (out_probe_ms) out_probe_ms[c] = 0.0;
    if (out_reps) out_reps[c] = 0;
    bool noop = false;
    gemm_status_t st = make_launch_args(config_ids[c], transA, transB, M, N, K, 1.f, A, lda, B, ldb, 0.f, C, ldc,
                                        batch, &args[c], &noop);
    if (st == GEMM_OK && noop) st = GEMM_ERR_INVALID_ARG;
    // A launch longer than kLongMs is its own warm-up; shorter ones are timed
    // again after `warmup` further launches.
    float ms = 0.f;
    for (int attempt = 0; attempt < 2 && st == GEMM_OK; ++attempt) {
      if (attempt == 1) {
        if (ms >= kLongMs) break;
        for (int w = 0; w < warmup && st == GEMM_OK; ++w) st = launch_by_id(config_ids[c], args[c], s);
        if (st != GEMM_OK) break;
      }
      cudaEventRecord(e0, s);
      st = launch_by_id(config_ids[c], args[c], s);
      cudaEventRecord(e1, s);
      cudaError_t ce = cudaEventSynchronize(e1);
      if (ce != cudaSuccess) {
        set_last_cuda_error(ce);
        st = GEMM_ERR_CUDA;
      }
      if (st == GEMM_OK) cudaEventElapsedTime(&ms, e0, e1);
    }
    out_status[c] = st;
    if (st == GEMM_OK) {
      out_ms[c] = ms;
      if (out_probe_ms) out_probe_ms[c] = ms;
      if (out_reps) out_reps[c] = 1;
      best = std::min(best, (double)ms);
    } else if (st == GEMM_ERR_CUDA) {
      ret = GEMM_ERR_CUDA;  // the context may be unusable: stop the sweep
    }
  }
  // Pass 2: back-to-back timed runs of the near-best configurations.
  for (int c = 0; c < n_configs && ret == GEMM_OK; ++c) {
    if (out_status[c] != GEMM_OK || out_ms[c] > refine_ratio * best) continue;
    const double probe = out_ms[c];
    int reps = probe > 0 ? (int)std::ceil(min_total_ms / probe) : max_reps;
    reps = std::max(min_reps, std::min(max_reps, reps));
    cudaEventRecord(e0, s);
    gemm_status_t st = GEMM_OK;
    for (int r = 0; r < reps && st == GEMM_OK; ++r) st = launch_by_id(config_ids[c], args[c], s);
    cudaEventRecord(e1, s);
    cudaError_t ce = cudaEventSynchronize(e1);
    if (ce != cudaSuccess) {
      set_last_cuda_error(ce);
      ret = GEMM_ERR_CUDA;
      break;
    }
    if (st != GEMM_OK) {
      out_status[c] = st;
      out_ms[c] = 0.0;
      continue;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    out_ms[c] = (double)ms / reps;
    if (out_reps) out_reps[c] = reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ret;
}
