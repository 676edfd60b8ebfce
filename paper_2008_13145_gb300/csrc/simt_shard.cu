// One shard of the FP32 SIMT instantiations.  This file is compiled
// kSimtShards times with -DKS_SHARD=<i>; shard i instantiates the config ids
// with (id / 2) % kSimtShards == i (each unstaged / staged pair together, so every
// shard holds the same mix of the costlier staged kernels), so the 576 kernels
// (and the 192 split-K instances) build in parallel.
#include <utility>

#include "simt_gemm.cuh"

#ifndef KS_SHARD
#error "compile with -DKS_SHARD=<shard index>"
#endif

namespace ks {
namespace {
#ifndef KS_SUBSET
#define KS_SUBSET 1  // debug builds instantiate every KS_SUBSET-th config only
#endif

template <int ID>
void reg_one(LaunchFn* table, LaunchFn* split, OccFn* occ) {
  if constexpr ((ID / 2) % kSimtShards == KS_SHARD && ID % KS_SUBSET == 0) {
    table[ID] = &launch_simt<ID, false>;
    if constexpr (split_eligible(ID)) {
      split[ID] = &launch_simt<ID, true>;
      occ[ID] = &occupancy_simt<ID>;
    }
  }
}
template <int... I>
void reg_all(std::integer_sequence<int, I...>, LaunchFn* table, LaunchFn* split, OccFn* occ) {
  (reg_one<I>(table, split, occ), ...);
}
}  // namespace

#define KS_CAT2(a, b) a##b
#define KS_CAT(a, b) KS_CAT2(a, b)
void KS_CAT(simt_register_shard_, KS_SHARD)(LaunchFn* table, LaunchFn* split, OccFn* occ) {
  reg_all(std::make_integer_sequence<int, kSimtConfigs>{}, table, split, occ);
}
}  // namespace ks
