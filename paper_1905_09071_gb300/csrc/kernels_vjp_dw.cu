// FFT kernels of the vector-Jacobian product, double-word FP32 path.
#include "launch.h"
#include "vjp_kernels.cuh"

namespace sag {

cudaError_t launch_k_fwd_col_dw(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st,
                                int base, int blocks, int all);

cudaError_t launch_vjp_fft_dw(const RhsParams& P, const LaunchCfg& L, const double* n, const double* g,
                              cudaStream_t st) {
  cudaError_t e = launch_k_fwd_col_dw(P, L, n, st, 0, L.col_blocks_all, 1);
  if (e != cudaSuccess) return e;
  k_gcol<cdw><<<L.inv_blocks, kThreads, L.vcol_smem, st>>>(P, g);
  k_rows_vjp<cdw><<<L.row_blocks, kThreads, L.vrow_smem, st>>>(P);
  k_inv_col_vjp<cdw><<<L.col_blocks_all, kThreads, L.vcol_smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t setup_vjp_fft_dw(const LaunchCfg& L) {
  (void)L;
  cudaError_t e = allow_max_smem(k_gcol<cdw>);
  if (e == cudaSuccess) e = allow_max_smem(k_rows_vjp<cdw>);
  if (e == cudaSuccess) e = allow_max_smem(k_inv_col_vjp<cdw>);
  return e;
}

}  // namespace sag
