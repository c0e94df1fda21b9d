// FFT stage of the FP64 path (runtime-length kernels only).
#include "tt_launch.cuh"

namespace sag {

cudaError_t enqueue_fft_f64(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st,
                            LaunchHook* hook) {
  if (hook) hook->mark(KID_FWD_COL, st);
  k_fwd_col<cd><<<L.col_blocks, kThreads, L.col_smem, st>>>(P, nin);
  if (L.has_tt) {
    cudaError_t e = launch_tt_stage<cd>(P, L, st, hook);
    if (e != cudaSuccess) return e;
  } else {
    if (hook) hook->mark(KID_ROWS, st);
    k_rows<cd><<<L.row_blocks, kThreads, L.row_smem, st>>>(P);
  }
  if (hook) hook->mark(KID_INV_COL, st);
  k_inv_col<cd><<<L.inv_blocks, kThreads, L.inv_smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_fwd_col_f64(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st) {
  k_fwd_col<cd><<<L.col_blocks, kThreads, L.col_smem, st>>>(P, nin);
  return cudaGetLastError();
}

cudaError_t setup_fft_kernels_f64(const LaunchCfg& L) {
  cudaError_t e = allow_max_smem(k_fwd_col<cd>);
  if (e == cudaSuccess) e = allow_max_smem(k_rows<cd>);
  if (e == cudaSuccess) e = allow_max_smem(k_inv_col<cd>);
  if (e == cudaSuccess) e = setup_tt_stage<cd>(L);
  return e;
}

}  // namespace sag
