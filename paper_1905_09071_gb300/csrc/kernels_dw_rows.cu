// k_rows for a double-word FP32 path (own translation unit: the
// compile-time length variants make it the slowest file to compile). The
// element type is SAG_DW_C: cdw here, cdwx in kernels_dwx_rows.cu. Each run of
// row blocks of one specialisation (KIND, fft_ct.cuh) gets its own
// instantiation.
#include <array>
#include <utility>

#include "fft_kernels.cuh"
#include "launch.h"

#ifndef SAG_DW_C
#define SAG_DW_C cdw
#endif

namespace sag {

namespace {

// Row specialisations that exist: the runtime-length path, the staged
// compile-time path for M2 = 64, 128, 256, 512 and the pair form for rows of
// 128, 256, 512 points; other kinds never occur and map to kKindGeneral.
constexpr bool row_kind(int K) {
  return K == kKindGeneral || K == kKindRuntime || K == kKindCt + 0 || K == kKindCt + 2 || K == kKindCt + 4 ||
         K == kKindCt + 6 || K == kKindPair + 2 || K == kKindPair + 4 || K == kKindPair + 6;
}

using RowLaunch = void (*)(const RhsParams&, int, int, size_t, cudaStream_t);
using Setup = cudaError_t (*)();

template <int K>
void row_kind_launch(const RhsParams& P, int base, int blocks, size_t smem, cudaStream_t st) {
  k_rows<SAG_DW_C, row_kind(K) ? K : kKindGeneral><<<blocks, kThreads, smem, st>>>(P, base);
}
template <int K>
cudaError_t row_setup() {
  return allow_max_smem(k_rows<SAG_DW_C, row_kind(K) ? K : kKindGeneral>);
}
template <int... K>
constexpr std::array<RowLaunch, sizeof...(K)> row_launches(std::integer_sequence<int, K...>) {
  return {{&row_kind_launch<K>...}};
}
template <int... K>
constexpr std::array<Setup, sizeof...(K)> row_setups(std::integer_sequence<int, K...>) {
  return {{&row_setup<K>...}};
}
constexpr auto kRows = row_launches(std::make_integer_sequence<int, kKindCount>{});
constexpr auto kRowSetup = row_setups(std::make_integer_sequence<int, kKindCount>{});

}  // namespace

cudaError_t launch_k_rows_dw(const RhsParams& P, const LaunchCfg& L, cudaStream_t st, int base, int blocks,
                             SAG_DW_C) {
  return for_kind_runs(L.row, base, base + blocks, [&](int kind, int b0, int b1) {
    kRows[kind](P, b0, b1 - b0, L.row_smem_kind[kind] ? L.row_smem_kind[kind] : L.row_smem, st);
    return cudaGetLastError();
  });
}

cudaError_t setup_k_rows_dw(const LaunchCfg& L, SAG_DW_C) {
  (void)L;
  for (Setup s : kRowSetup) {
    const cudaError_t e = s();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sag
