// Instantiation of the FFT kernels for the double-word FP32 path.
#include "fft_kernels.cuh"
#include "launch.h"

namespace sag {

cudaError_t enqueue_fft_dw(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st,
                           LaunchHook* hook) {
  if (hook) hook->mark(KID_FWD_COL, st);
  k_fwd_col<cdw><<<L.col_blocks, kThreads, L.col_smem, st>>>(P, nin);
  if (hook) hook->mark(KID_ROWS, st);
  k_rows<cdw><<<L.row_blocks, kThreads, L.row_smem, st>>>(P);
  if (hook) hook->mark(KID_INV_COL, st);
  k_inv_col<cdw><<<L.inv_blocks, kThreads, L.inv_smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t setup_fft_kernels_dw(const LaunchCfg& L) {
  cudaError_t e = cudaFuncSetAttribute(k_fwd_col<cdw>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.col_smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rows<cdw>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.row_smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inv_col<cdw>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.inv_smem);
  return e;
}

}  // namespace sag
