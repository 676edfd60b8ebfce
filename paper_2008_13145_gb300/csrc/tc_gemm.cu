// Tensor-core GEMM families (tcgen05 + TMA + TMEM) -- config space.
#include <cstring>

#include "common.cuh"

namespace ks {
namespace {
constexpr int kTcBn[3] = {64, 128, 256};
constexpr int kTcStages[3] = {2, 3, 4};
}  // namespace

bool tc_config_valid(int id) {
  const int fam = (id - kTcBase) / 100, idx = (id - kTcBase) % 100;
  return id >= kTcBase && fam >= 0 && fam < 3 && idx < kTcConfigsPerFamily;
}

gemm_status_t tc_params(int id, int32_t out[8]) {
  if (!tc_config_valid(id)) return GEMM_ERR_NO_KERNEL;
  const int fam = (id - kTcBase) / 100 + 1, idx = (id - kTcBase) % 100;
  const int bk = (fam == GEMM_PREC_TF32) ? 32 : 64;
  int32_t v[8] = {fam, 128, kTcBn[idx / 6], bk, kTcStages[(idx / 2) % 3], idx % 2, 0, 0};
  std::memcpy(out, v, sizeof(v));
  return GEMM_OK;
}

gemm_status_t tc_launch(int, const GemmArgs&, cudaStream_t) { return GEMM_ERR_UNSUPPORTED; }
}  // namespace ks
