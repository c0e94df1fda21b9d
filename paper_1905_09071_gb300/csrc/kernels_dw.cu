// FFT stage of the double-word FP32 path: the kernels live in their own
// translation units (kernels_dw_{fwd,rows,inv,tt}.cu).
#include "launch.h"

namespace sag {

cudaError_t launch_k_fwd_col_dw(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st,
                                int base, int blocks, int all);
cudaError_t launch_k_rows_dw(const RhsParams& P, const LaunchCfg& L, cudaStream_t st, int base, int blocks);
cudaError_t launch_k_inv_col_dw(const RhsParams& P, const LaunchCfg& L, cudaStream_t st, int base, int blocks);
cudaError_t launch_tt_dw(const RhsParams& P, const LaunchCfg& L, cudaStream_t st, LaunchHook* hook);
cudaError_t setup_k_fwd_col_dw(const LaunchCfg& L);
cudaError_t setup_k_rows_dw(const LaunchCfg& L);
cudaError_t setup_k_inv_col_dw(const LaunchCfg& L);
cudaError_t setup_tt_dw(const LaunchCfg& L);

cudaError_t enqueue_fft_dw(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st,
                           LaunchHook* hook, const FftRange* r) {
  const FftRange all{0, L.col_blocks, 0, L.row_blocks, 0, L.inv_blocks};
  const FftRange& R = r ? *r : all;
  if (hook) hook->mark(KID_FWD_COL, st);
  cudaError_t e = launch_k_fwd_col_dw(P, L, nin, st, R.col0, R.col1 - R.col0, 0);
  if (e != cudaSuccess) return e;
  if (L.has_tt) {
    if ((e = launch_tt_dw(P, L, st, hook)) != cudaSuccess) return e;  // every item (no groups with TT)
  } else {
    if (hook) hook->mark(KID_ROWS, st);
    if ((e = launch_k_rows_dw(P, L, st, R.row0, R.row1 - R.row0)) != cudaSuccess) return e;
  }
  if (hook) hook->mark(KID_INV_COL, st);
  return launch_k_inv_col_dw(P, L, st, R.inv0, R.inv1 - R.inv0);
}

cudaError_t setup_fft_kernels_dw(const LaunchCfg& L) {
  cudaError_t e = setup_k_fwd_col_dw(L);
  if (e == cudaSuccess) e = setup_k_rows_dw(L);
  if (e == cudaSuccess) e = setup_k_inv_col_dw(L);
  if (e == cudaSuccess) e = setup_tt_dw(L);
  return e;
}

}  // namespace sag
