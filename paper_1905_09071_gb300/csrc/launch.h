// Host-side launch interface between the ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "plan.h"

namespace sag {

// Grid and shared-memory sizes of one plan, computed once at plan time.
// The entries of one block table (items in table order) with the kernel
// specialisation (KIND, fft_ct.cuh) each entry's blocks run.
struct KindTable {
  const int* pre = nullptr;   // [n + 1] block prefix (host copy)
  const int* kind = nullptr;  // [n] specialisation of each entry
  int n = 0;
};

struct LaunchCfg {
  KindTable col, col_all, row;  // forward columns (pairs or distinct vectors; every vector), rows
  int prep_blocks;
  int col_blocks, row_blocks, inv_blocks, epi_blocks;
  int col_blocks_all;  // column blocks over every vector (the adjoint's passes)
  int chain_blocks;
  int ent_blocks;       // TT adjoint: inverse column blocks over every core entry
  int has_tt;           // the plan's systems use TT kernels (one format per plan)
  int vjp_rmax;         // largest CP rank of an item: the adjoint row pass's grid height
  size_t col_smem, row_smem, inv_smem, epi_smem, coef_smem, rowtt_smem;
  size_t col_smem_kind[kKindCount], row_smem_kind[kKindCount];  // per kernel specialisation
  size_t vcol_smem, vrow_smem;  // vector-Jacobian product kernels (0: not available)
};

// What the epilogue writes (see EpiMode).
struct EpiArgs {
  const double* nin;    // state the right-hand side is evaluated at
  double* nbase;        // RK2 base state (updated in place by the second stage)
  double* out0;         // EPI_RHS: dn/dt; first stages: the intermediate state
  double* pout;         // EPI_RHS: gain part (nullable)
  double* qout;         // EPI_RHS: loss part (nullable)
  double* k1buf;        // Heun: F at the first stage
  double* diag;         // second stages: [steps+1][3] diagnostics (nullable)
  double* outflow_out;  // EPI_RHS: outflow (nullable, device)
  double* part;         // [epi_blocks][4] block partials
  double dt;
  int mode;
  int flux;             // 1: compute the outflow (diag or outflow_out wanted)
  int split_next;       // first stages (double-word path): also write out0's double-word copy
  int presplit;         // the double-word copy of nin is current: skip k_nmax and k_nsplit
};

// Kernel ids for profiling (order of sag_kernel_name).
enum KernelId : int {
  KID_NMAX = 0, KID_NSPLIT = 1, KID_DOT = 2, KID_FWD_COL = 3, KID_ROWS = 4, KID_INV_COL = 5,
  KID_EPILOGUE = 6, KID_MOMENTS = 7, KID_COEF = 8, KID_ROWS_TT = 9, KID_TT_CHAIN = 10,
  KID_ROWS_TT_INV = 11, KID_QTERM = 12, KID_COUNT = 13
};

// Splits the blocks [b0, b1) of table t into runs of equal specialisation
// and calls launch(kind, r0, r1) for each; with more than kMaxKindRuns runs
// it launches the run-time dispatching kernel over the whole range instead
// (kind kKindGeneral). Plans whose items alternate between many kinds (a
// batch of systems with mixed lengths) order their block tables by kind
// (kind_order), so that they stay within one run per kind.
constexpr int kMaxKindRuns = kKindCount;
template <class F>
cudaError_t for_kind_runs(const KindTable& t, int b0, int b1, F&& launch) {
  if (b1 <= b0) return cudaSuccess;
  int rk[kMaxKindRuns], r0[kMaxKindRuns], r1[kMaxKindRuns], nr = 0;
  bool general = t.kind == nullptr;
  for (int i = 0; i < t.n && !general; ++i) {
    const int a = t.pre[i] > b0 ? t.pre[i] : b0, z = t.pre[i + 1] < b1 ? t.pre[i + 1] : b1;
    if (a >= z) continue;
    if (nr > 0 && rk[nr - 1] == t.kind[i] && r1[nr - 1] == a) {
      r1[nr - 1] = z;
      continue;
    }
    if (nr == kMaxKindRuns) {
      general = true;
      break;
    }
    rk[nr] = t.kind[i];
    r0[nr] = a;
    r1[nr] = z;
    ++nr;
  }
  if (general) return launch(kKindGeneral, b0, b1);
  for (int r = 0; r < nr; ++r) {
    const cudaError_t e = launch(rk[r], r0[r], r1[r]);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Order of a block table's entries: the identity when kinds[] (in item order)
// forms at most kMaxKindRuns runs of equal kind, else the items stably sorted
// by kind. Returns whether it sorted.
inline bool kind_order(const int* kinds, int n, int* order) {
  int runs = 0;
  for (int i = 0; i < n; ++i) {
    order[i] = i;
    runs += (i == 0 || kinds[i] != kinds[i - 1]);
  }
  if (runs <= kMaxKindRuns) return false;
  std::stable_sort(order, order + n, [&](int a, int b) { return kinds[a] < kinds[b]; });
  return true;
}

// Optional hook called before each kernel launch (id) and once after the last
// one (id = -1), on the launch stream.
struct LaunchHook {
  virtual void mark(int id, cudaStream_t st) = 0;
  virtual ~LaunchHook() = default;
};

// A second stream with fork/join events: the FP64 inner products run on it,
// beside the FFT kernels (also inside a captured graph, as a parallel branch).
struct SideStream {
  cudaStream_t stream;
  cudaEvent_t fork, join;
};

// Block ranges [begin, end) of the three FFT kernels' tables (colpre, rowpre in
// rowperm order, invpre) for one group of items.
struct FftRange {
  int col0, col1, row0, row1, inv0, inv1;
};

// FFT groups run on their own streams (graph branches) so that one order's
// ALU-heavy row pass overlaps another order's memory-heavy column pass.
constexpr int kMaxFftGroups = 4;
struct FftGroups {
  int n;                            // 0: one launch per kernel on the caller's stream
  FftRange r[kMaxFftGroups];
  SideStream s[kMaxFftGroups];      // stream, and the events that fork and join it
};

cudaError_t enqueue_eval(const RhsParams& P, const LaunchCfg& L, const double* nin,
                         const EpiArgs& A, cudaStream_t st, LaunchHook* hook = nullptr,
                         const SideStream* side = nullptr, const FftGroups* groups = nullptr);
// Largest dynamic shared memory a block may use on the current device.
inline int smem_limit() {
  int dev = 0, v = 48 * 1024;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

// Lets `func` use all the dynamic shared memory its static shared memory
// leaves free. The attribute is per function for the whole process, so a
// per-plan value would shrink the limit of plans built earlier. A template
// kernel instantiated in several translation units is a separate function in
// each (its host stub has internal linkage): the file that launches it must
// set the attribute on its own copy, or launch through a function of the file
// that does.
template <class F>
inline cudaError_t allow_max_smem(F* func) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, func);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_limit() - (int)a.sharedSizeBytes);
}

cudaError_t enqueue_moments(const RhsParams& P, const double* n, double* diag, cudaStream_t st);
// FFT stage over the block range r (nullptr: every item).
cudaError_t enqueue_fft_f64(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st,
                            LaunchHook* hook, const FftRange* r = nullptr);
cudaError_t enqueue_fft_dw(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st,
                           LaunchHook* hook, const FftRange* r = nullptr);
cudaError_t setup_common_kernels(const LaunchCfg& L);
// n -> double-word with its per-system power-of-two scale (resets nothing).
cudaError_t enqueue_nsplit(const RhsParams& P, const LaunchCfg& L, const double* n, cudaStream_t st);
// Vector-Jacobian product of the CP right-hand side at n for cotangent g:
// gn = (dF/dn)^T g, gU (vector layout) = (dF/dU)^T g, added to gU if accumulate.
// With side, the product rule's inner products run on side->stream (forked
// and joined inside the call).
cudaError_t enqueue_vjp(const RhsParams& P, const LaunchCfg& L, const double* n, const double* g,
                        double* gn, double* gU, int accumulate, cudaStream_t st,
                        const SideStream* side = nullptr);
cudaError_t enqueue_axpby(double* out, double a, const double* x, double b, const double* y, int64_t n,
                          cudaStream_t st);
// u i^a for i = 1..N by the parametric factors' generator (sag_power_eval).
cudaError_t enqueue_power_eval(float4 up, const float2* lnt, const float* ek, int N, double* out, cudaStream_t st);
// One RK2 stage from a given right-hand side k (sag_rk2_stage).
cudaError_t enqueue_rk2_stage(const RhsParams& P, int stage, int midpoint, double* n, double* nstar,
                              double* k1, const double* k, double dt, cudaStream_t st);
cudaError_t setup_vjp_common(const LaunchCfg& L);
cudaError_t setup_vjp_fft_f64(const LaunchCfg& L);
cudaError_t setup_fft_kernels_f64(const LaunchCfg& L);
// Both double-word paths' FFT and adjoint kernels.
cudaError_t setup_fft_kernels_dw(const LaunchCfg& L);

// Double-word kernels per element type: cdw (grid-aligned butterflies,
// kernels_dw_*.cu) and cdwx (plain double-word, kernels_dwx_*.cu); the last
// argument only selects the type.
#define SAG_DW_DECLS(C)                                                                                    \
  cudaError_t launch_k_fwd_col_dw(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st, \
                                  int base, int blocks, int all, C);                                     \
  cudaError_t launch_k_rows_dw(const RhsParams& P, const LaunchCfg& L, cudaStream_t st, int base, int blocks, \
                               C);                                                                       \
  cudaError_t launch_k_inv_col_dw(const RhsParams& P, const LaunchCfg& L, cudaStream_t st, int base,        \
                                  int blocks, C);                                                        \
  cudaError_t launch_tt_dw(const RhsParams& P, const LaunchCfg& L, cudaStream_t st, LaunchHook* hook, C);  \
  cudaError_t launch_vjp_fft_dw(const RhsParams& P, const LaunchCfg& L, const double* n, const double* g,  \
                                cudaStream_t st, C);                                                     \
  cudaError_t launch_vjp_fft_tt_dw(const RhsParams& P, const LaunchCfg& L, const double* n,               \
                                   const double* g, cudaStream_t st, C);                                \
  cudaError_t setup_k_fwd_col_dw(const LaunchCfg& L, C);                                                 \
  cudaError_t setup_k_rows_dw(const LaunchCfg& L, C);                                                    \
  cudaError_t setup_k_inv_col_dw(const LaunchCfg& L, C);                                                 \
  cudaError_t setup_tt_dw(const LaunchCfg& L, C);                                                        \
  cudaError_t setup_vjp_fft_dw(const LaunchCfg& L, C);
SAG_DW_DECLS(cdw)
SAG_DW_DECLS(cdwx)
#undef SAG_DW_DECLS

}  // namespace sag
