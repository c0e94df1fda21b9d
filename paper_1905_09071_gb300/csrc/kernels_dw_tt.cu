// TT stage of the double-word FP32 path.
#include "tt_launch.cuh"

namespace sag {

cudaError_t launch_tt_dw(const RhsParams& P, const LaunchCfg& L, cudaStream_t st, LaunchHook* hook) {
  return launch_tt_stage<cdw>(P, L, st, hook);
}

cudaError_t setup_tt_dw(const LaunchCfg& L) { return setup_tt_stage<cdw>(L); }

}  // namespace sag
