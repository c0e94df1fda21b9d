// FFT stage of the FP64 path (runtime-length kernels only).
#include "tt_launch.cuh"

namespace sag {

cudaError_t enqueue_fft_f64(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st,
                            LaunchHook* hook, const FftRange* r) {
  const FftRange all{0, L.col_blocks, 0, L.row_blocks, 0, L.inv_blocks};
  const FftRange& R = r ? *r : all;
  if (hook) hook->mark(KID_FWD_COL, st);
  if (R.col1 > R.col0) k_fwd_col<cd><<<R.col1 - R.col0, kThreads, L.col_smem, st>>>(P, nin, R.col0, 0);
  if (L.has_tt) {
    cudaError_t e = launch_tt_stage<cd>(P, L, st, hook);  // every item (no groups with TT)
    if (e != cudaSuccess) return e;
  } else {
    if (hook) hook->mark(KID_ROWS, st);
    if (R.row1 > R.row0) k_rows<cd><<<R.row1 - R.row0, kThreads, L.row_smem, st>>>(P, R.row0);
  }
  if (hook) hook->mark(KID_INV_COL, st);
  if (R.inv1 > R.inv0) k_inv_col<cd><<<R.inv1 - R.inv0, kThreads, L.inv_smem, st>>>(P, R.inv0);
  return cudaGetLastError();
}

// Forward columns for the vector-Jacobian products: blocks of the core or
// rank vectors (all = 0, as in the right-hand side) or of every vector
// (all = 1). Launched from this file because the shared-memory attribute
// belongs to this file's copy of the kernel.
cudaError_t launch_fwd_col_f64(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st,
                               int blocks, int all) {
  if (blocks > 0) k_fwd_col<cd><<<blocks, kThreads, L.col_smem, st>>>(P, nin, 0, all);
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
