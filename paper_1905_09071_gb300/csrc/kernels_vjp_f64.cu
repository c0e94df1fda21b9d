// FFT kernels of the vector-Jacobian product, FP64 path.
#include "launch.h"
#include "vjp_kernels.cuh"
#include "vjp_tt.cuh"

namespace sag {

cudaError_t launch_fwd_col_f64(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st,
                               int blocks, int all);

cudaError_t launch_vjp_fft_f64(const RhsParams& P, const LaunchCfg& L, const double* n, const double* g,
                              cudaStream_t st) {
  cudaError_t e = launch_fwd_col_f64(P, L, n, st, L.col_blocks_all, 1);
  if (e != cudaSuccess) return e;
  k_gcol<cd><<<L.inv_blocks, kThreads, L.vcol_smem, st>>>(P, g);
  k_rows_vjp<cd><<<dim3(L.row_blocks, L.vjp_rmax), kThreads, L.vrow_smem, st>>>(P);
  k_inv_col_vjp<cd><<<L.col_blocks_all, kThreads, L.vcol_smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_vjp_fft_tt_f64(const RhsParams& P, const LaunchCfg& L, const double* n, const double* g,
                                  cudaStream_t st) {
  cudaError_t e = launch_fwd_col_f64(P, L, n, st, L.col_blocks, 0);
  if (e != cudaSuccess) return e;
  return launch_vjp_tt_after_cols<cd>(P, L, g, st);
}

cudaError_t setup_vjp_fft_f64(const LaunchCfg& L) {
  (void)L;
  cudaError_t e = allow_max_smem(k_gcol<cd>);
  if (e == cudaSuccess) e = allow_max_smem(k_rows_vjp<cd>);
  if (e == cudaSuccess) e = allow_max_smem(k_inv_col_vjp<cd>);
  if (e == cudaSuccess) e = setup_vjp_tt<cd>(L);
  return e;
}

}  // namespace sag
