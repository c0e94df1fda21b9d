// FFT kernels of the vector-Jacobian product, a double-word FP32 path;
// element type SAG_DW_C (cdw here, cdwx in kernels_vjp_dwx.cu).
#include "launch.h"
#include "vjp_kernels.cuh"
#include "vjp_tt.cuh"

#ifndef SAG_DW_C
#define SAG_DW_C cdw
#endif

namespace sag {

cudaError_t launch_vjp_fft_dw(const RhsParams& P, const LaunchCfg& L, const double* n, const double* g,
                              cudaStream_t st, SAG_DW_C) {
  cudaError_t e = launch_k_fwd_col_dw(P, L, n, st, 0, L.col_blocks_all, 1, SAG_DW_C{});
  if (e != cudaSuccess) return e;
  k_gcol<SAG_DW_C><<<L.inv_blocks, kThreads, L.vcol_smem, st>>>(P, g);
  k_rows_vjp<SAG_DW_C><<<dim3(L.row_blocks, L.vjp_rmax), kThreads, L.vrow_smem, st>>>(P);
  k_inv_col_vjp<SAG_DW_C><<<L.col_blocks_all, kThreads, L.vcol_smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_vjp_fft_tt_dw(const RhsParams& P, const LaunchCfg& L, const double* n, const double* g,
                                 cudaStream_t st, SAG_DW_C) {
  cudaError_t e = launch_k_fwd_col_dw(P, L, n, st, 0, L.col_blocks, 0, SAG_DW_C{});
  if (e != cudaSuccess) return e;
  return launch_vjp_tt_after_cols<SAG_DW_C>(P, L, g, st);
}

cudaError_t setup_vjp_fft_dw(const LaunchCfg& L, SAG_DW_C) {
  (void)L;
  cudaError_t e = allow_max_smem(k_gcol<SAG_DW_C>);
  if (e == cudaSuccess) e = allow_max_smem(k_rows_vjp<SAG_DW_C>);
  if (e == cudaSuccess) e = allow_max_smem(k_inv_col_vjp<SAG_DW_C>);
  if (e == cudaSuccess) e = setup_vjp_tt<SAG_DW_C>(L);
  return e;
}

}  // namespace sag
