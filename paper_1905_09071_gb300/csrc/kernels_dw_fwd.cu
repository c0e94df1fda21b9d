// k_fwd_col for the double-word FP32 path (own translation unit: the
// compile-time length variants make it the slowest file to compile).
#include "fft_kernels.cuh"
#include "launch.h"

namespace sag {

cudaError_t launch_k_fwd_col_dw(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st,
                                int base, int blocks, int all) {
  if (blocks > 0) k_fwd_col<cdw><<<blocks, kThreads, L.col_smem, st>>>(P, nin, base, all);
  return cudaGetLastError();
}

cudaError_t setup_k_fwd_col_dw(const LaunchCfg& L) {
  return allow_max_smem(k_fwd_col<cdw>);
}

}  // namespace sag
