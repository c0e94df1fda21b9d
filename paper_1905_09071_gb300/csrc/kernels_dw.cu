// FFT stage of the double-word FP32 paths: the kernels live in their own
// translation units (kernels_dw_{fwd,rows,inv,tt}.cu for cdw, the
// grid-aligned butterflies; kernels_dwx_*.cu for cdwx, plain double-word).
// P.exact picks the path.
#include "launch.h"

namespace sag {

namespace {

template <class C>
cudaError_t enqueue_fft_dwc(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st,
                            LaunchHook* hook, const FftRange* r) {
  const FftRange all{0, L.col_blocks, 0, L.row_blocks, 0, L.inv_blocks};
  const FftRange& R = r ? *r : all;
  if (hook) hook->mark(KID_FWD_COL, st);
  cudaError_t e = launch_k_fwd_col_dw(P, L, nin, st, R.col0, R.col1 - R.col0, 0, C{});
  if (e != cudaSuccess) return e;
  if (L.has_tt) {
    if ((e = launch_tt_dw(P, L, st, hook, C{})) != cudaSuccess) return e;  // every item (no groups with TT)
  } else {
    if (hook) hook->mark(KID_ROWS, st);
    if ((e = launch_k_rows_dw(P, L, st, R.row0, R.row1 - R.row0, C{})) != cudaSuccess) return e;
  }
  if (hook) hook->mark(KID_INV_COL, st);
  return launch_k_inv_col_dw(P, L, st, R.inv0, R.inv1 - R.inv0, C{});
}

template <class C>
cudaError_t setup_fft_dwc(const LaunchCfg& L) {
  cudaError_t e = setup_k_fwd_col_dw(L, C{});
  if (e == cudaSuccess) e = setup_k_rows_dw(L, C{});
  if (e == cudaSuccess) e = setup_k_inv_col_dw(L, C{});
  if (e == cudaSuccess) e = setup_tt_dw(L, C{});
  if (e == cudaSuccess) e = setup_vjp_fft_dw(L, C{});
  return e;
}

}  // namespace

cudaError_t enqueue_fft_dw(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st,
                           LaunchHook* hook, const FftRange* r) {
  return P.exact ? enqueue_fft_dwc<cdwx>(P, L, nin, st, hook, r) : enqueue_fft_dwc<cdw>(P, L, nin, st, hook, r);
}

cudaError_t launch_vjp_fft_dw(const RhsParams& P, const LaunchCfg& L, const double* n, const double* g,
                              cudaStream_t st) {
  return P.exact ? launch_vjp_fft_dw(P, L, n, g, st, cdwx{}) : launch_vjp_fft_dw(P, L, n, g, st, cdw{});
}

cudaError_t launch_vjp_fft_tt_dw(const RhsParams& P, const LaunchCfg& L, const double* n, const double* g,
                                 cudaStream_t st) {
  return P.exact ? launch_vjp_fft_tt_dw(P, L, n, g, st, cdwx{}) : launch_vjp_fft_tt_dw(P, L, n, g, st, cdw{});
}

cudaError_t setup_fft_kernels_dw(const LaunchCfg& L) {
  cudaError_t e = setup_fft_dwc<cdw>(L);
  if (e == cudaSuccess) e = setup_fft_dwc<cdwx>(L);
  return e;
}

}  // namespace sag
