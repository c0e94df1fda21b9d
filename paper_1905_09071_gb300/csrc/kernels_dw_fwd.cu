// k_fwd_col for a double-word FP32 path (own translation unit: the
// compile-time length variants make it the slowest file to compile). The
// element type is SAG_DW_C: cdw here, cdwx in kernels_dwx_fwd.cu. Each run of
// column blocks of one specialisation (KIND, fft_ct.cuh) gets its own
// instantiation.
#include <array>
#include <utility>

#include "fft_kernels.cuh"
#include "launch.h"

#ifndef SAG_DW_C
#define SAG_DW_C cdw
#define SAG_DW_GEN 1  // the generating variants exist for this element type only
#endif
#ifndef SAG_DW_GEN
#define SAG_DW_GEN 0
#endif

namespace sag {

namespace {

using FwdLaunch = void (*)(const RhsParams&, const double*, int, int, int, size_t, cudaStream_t);
using Setup = cudaError_t (*)();

// The pair form exists for column lengths up to 1024 (its rows are at most 512
// points, so the 1536-point columns never pair); that kind maps to kKindGeneral.
constexpr int fwd_kind_of(int K) { return K == kKindPair + ct_index(1536) ? kKindGeneral : K; }

// GEN: plans of parametric factors generate u i^a in the loads (a separate
// instantiation of every kind).
template <int K, bool GEN>
void fwd_kind(const RhsParams& P, const double* nin, int base, int blocks, int all, size_t smem,
              cudaStream_t st) {
  k_fwd_col<SAG_DW_C, fwd_kind_of(K), GEN><<<blocks, kThreads, smem, st>>>(P, nin, base, all);
}
template <int K, bool GEN>
cudaError_t fwd_setup() {
  return allow_max_smem(k_fwd_col<SAG_DW_C, fwd_kind_of(K), GEN>);
}
template <bool GEN, int... K>
constexpr std::array<FwdLaunch, sizeof...(K)> fwd_launches(std::integer_sequence<int, K...>) {
  return {{&fwd_kind<K, GEN>...}};
}
template <bool GEN, int... K>
constexpr std::array<Setup, sizeof...(K)> fwd_setups(std::integer_sequence<int, K...>) {
  return {{&fwd_setup<K, GEN>...}};
}
constexpr auto kFwd = fwd_launches<false>(std::make_integer_sequence<int, kKindCount>{});
constexpr auto kFwdSetup = fwd_setups<false>(std::make_integer_sequence<int, kKindCount>{});
#if SAG_DW_GEN
constexpr auto kFwdGen = fwd_launches<true>(std::make_integer_sequence<int, kKindCount>{});
constexpr auto kFwdGenSetup = fwd_setups<true>(std::make_integer_sequence<int, kKindCount>{});
#endif

}  // namespace

cudaError_t launch_k_fwd_col_dw(const RhsParams& P, const LaunchCfg& L, const double* nin, cudaStream_t st,
                                int base, int blocks, int all, SAG_DW_C) {
#if SAG_DW_GEN
  const auto& table = P.vpow ? kFwdGen : kFwd;
#else
  const auto& table = kFwd;  // plans of parametric factors read the stored copy on this path
#endif
  return for_kind_runs(all ? L.col_all : L.col, base, base + blocks, [&](int kind, int b0, int b1) {
    table[kind](P, nin, b0, b1 - b0, all, L.col_smem_kind[kind] ? L.col_smem_kind[kind] : L.col_smem, st);
    return cudaGetLastError();
  });
}

cudaError_t setup_k_fwd_col_dw(const LaunchCfg& L, SAG_DW_C) {
  (void)L;
  for (Setup s : kFwdSetup) {
    const cudaError_t e = s();
    if (e != cudaSuccess) return e;
  }
#if SAG_DW_GEN
  for (Setup s : kFwdGenSetup) {
    const cudaError_t e = s();
    if (e != cudaSuccess) return e;
  }
#endif
  return cudaSuccess;
}

}  // namespace sag
