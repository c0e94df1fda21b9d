// k_inv_col for a double-word FP32 path (own translation unit: the
// compile-time length variants make it the slowest file to compile). The
// element type is SAG_DW_C: cdw here, cdwx in kernels_dwx_inv.cu. One launch
// covers every item (the run-time dispatching kernel): with about one block
// per SM, separate launches per length would run one after another.
#include "fft_kernels.cuh"
#include "launch.h"

#ifndef SAG_DW_C
#define SAG_DW_C cdw
#endif

namespace sag {

cudaError_t launch_k_inv_col_dw(const RhsParams& P, const LaunchCfg& L, cudaStream_t st, int base, int blocks,
                                SAG_DW_C) {
  if (blocks > 0) k_inv_col<SAG_DW_C><<<blocks, kThreads, L.inv_smem, st>>>(P, base);
  return cudaGetLastError();
}

cudaError_t setup_k_inv_col_dw(const LaunchCfg& L, SAG_DW_C) {
  (void)L;
  return allow_max_smem(k_inv_col<SAG_DW_C>);
}

}  // namespace sag
