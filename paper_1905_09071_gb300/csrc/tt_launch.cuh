// Launch of the TT stage (row spectra, per-frequency chain, inverse rows) for
// one complex scalar type; included by the translation unit of that type.
#pragma once

#include "fft_kernels.cuh"
#include "launch.h"

namespace sag {

template <class C>
cudaError_t launch_tt_stage(const RhsParams& P, const LaunchCfg& L, cudaStream_t st, LaunchHook* hook) {
  // (a plan whose every order is idle has no blocks at all)
  if (hook) hook->mark(KID_ROWS_TT, st);
  if (L.row_blocks > 0) k_rows_tt_fwd<C><<<L.row_blocks, kThreads, L.rowtt_smem, st>>>(P);
  if (hook) hook->mark(KID_TT_CHAIN, st);
  if (L.chain_blocks == 0) {
  } else if (P.tt_rmax <= 4) {
    k_tt_chain<C, 4><<<L.chain_blocks, 256, 0, st>>>(P);
  } else if (P.tt_rmax <= 8) {
    k_tt_chain<C, 8><<<L.chain_blocks, 256, 0, st>>>(P);
  } else {
    k_tt_chain<C, 16><<<L.chain_blocks, 256, 0, st>>>(P);
  }
  if (hook) hook->mark(KID_ROWS_TT_INV, st);
  if (L.row_blocks > 0) k_rows_tt_inv<C><<<L.row_blocks, kThreads, L.rowtt_smem, st>>>(P);
  return cudaGetLastError();
}

template <class C>
cudaError_t setup_tt_stage(const LaunchCfg& L) {
  cudaError_t e = allow_max_smem(k_rows_tt_fwd<C>);
  if (e == cudaSuccess)
    e = allow_max_smem(k_rows_tt_inv<C>);
  return e;
}

}  // namespace sag
