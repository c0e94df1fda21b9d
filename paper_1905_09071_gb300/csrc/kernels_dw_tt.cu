// TT stage of a double-word FP32 path; element type SAG_DW_C (cdw here, cdwx
// in kernels_dwx_tt.cu).
#include "tt_launch.cuh"

#ifndef SAG_DW_C
#define SAG_DW_C cdw
#endif

namespace sag {

cudaError_t launch_tt_dw(const RhsParams& P, const LaunchCfg& L, cudaStream_t st, LaunchHook* hook, SAG_DW_C) {
  return launch_tt_stage<SAG_DW_C>(P, L, st, hook);
}

cudaError_t setup_tt_dw(const LaunchCfg& L, SAG_DW_C) { return setup_tt_stage<SAG_DW_C>(L); }

}  // namespace sag
