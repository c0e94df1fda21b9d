// Host-side plan object shared by the plan builder (plan_build.cu) and the C
// ABI (api.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "launch.h"
#include "sag.h"

namespace sag {

sag_status fail(sag_status s, const std::string& msg);
sag_status cuda_fail(cudaError_t e, const char* where);

// Records one CUDA event before each kernel launch and one after the last.
struct EventHook : LaunchHook {
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, cudaEvent_t>> marks;
  bool failed = false;
  void mark(int id, cudaStream_t st) override;
  ~EventHook() override;
};

}  // namespace sag

struct sag_plan_s {
  sag::RhsParams P{};
  sag::LaunchCfg L{};
  int B = 0, prec = 0, rk = 0, sym = 1, fmt = 0;
  int64_t Ntot = 0;
  int64_t nfactor = 0;                    // factor values over all vectors (vector layout)
  int64_t nfactor_dw = 0;                 // length of the padded double-word factor copy
  // integrate_vjp buffers, allocated on first use
  double* vjp_pool = nullptr;
  size_t vjp_pool_len = 0;
  double* stage_g = nullptr;              // host-buffer staging of factor-sized arrays
  size_t stage_g_len = 0;
  std::vector<int64_t> offsets;           // [B + 1] packed offsets
  std::vector<sag::OrderDesc> items;      // host copy of the item table
  std::vector<sag::SysDesc> systems;      // host copy of the system table
  std::vector<void*> allocs;
  size_t bytes = 0;
  double* nstar = nullptr;
  double* k1buf = nullptr;
  double* epi_part = nullptr;
  double* stage_a = nullptr;   // host-buffer staging (inputs)
  double* stage_b = nullptr;   // host-buffer staging (outputs)
  double* stage_c = nullptr;
  double* dev_outflow = nullptr;
  double* stage_diag = nullptr;
  size_t stage_diag_len = 0;
  cudaStream_t cap_stream = nullptr;
  sag::SideStream side{nullptr, nullptr, nullptr};
  sag::FftGroups groups{};
  int fft_groups = 1;                     // stream groups of the FFT stage (1: one launch per kernel)
  std::vector<int> m2_pref;               // per item: M2 of its four-step split (0: the rule)
  bool col_sorted = false;                // column and row tables ordered by kernel kind (one FFT group)
  std::string tune_log;                   // candidates the geometry autotuner timed (JSON objects)
  std::vector<int> h_colpre, h_invpre;    // host copies of the block tables, for regrouping
  std::vector<int> h_colpre_all, h_rowpre, h_rowperm;
  std::vector<int> h_colkind, h_colkind_all, h_rowkind;  // kernel specialisations (LaunchCfg)
  std::vector<int> h_nrowpair;
  std::vector<int> h_umap, h_ulist;  // CP slot maps of repeated vectors (host copies)
  std::vector<double> h_work;             // FFT points per item, for balancing groups
  std::vector<int> h_nvec;                // vectors per item (row blocks go heaviest first)
  // SAG_CP_POWER plans: (u, a) of every vector in vector order; the forward
  // column kernels generate U = u i^a instead of reading it.
  std::vector<double> pow_ua;
  bool prof = false;
  sag::EventHook hook;
  // Instantiated graphs of sag_rhs / sag_rk2_step calls, keyed by the call's
  // kind, device pointers and dt (a few, most recent last).
  struct GraphKey {
    int kind;
    const void* p0;
    const void* p1;
    double dt;
    const void* p2 = nullptr;
    int64_t i0 = 0;
  };
  std::vector<std::pair<GraphKey, cudaGraphExec_t>> gcache;
  cudaGraphExec_t gexec = nullptr;
  const double* g_n = nullptr;
  double g_dt = 0.0;
  double* g_diag = nullptr;

  template <class T>
  cudaError_t alloc(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
    if (e != cudaSuccess) return e;
    allocs.push_back(q);
    bytes += count * sizeof(T);
    *p = static_cast<T*>(q);
    return cudaSuccess;
  }
  template <class T>
  cudaError_t upload(T** p, const std::vector<T>& h) {
    cudaError_t e = alloc(p, h.size() ? h.size() : 1);
    if (e != cudaSuccess || h.empty()) return e;
    return cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  }
  ~sag_plan_s() {
    if (gexec) cudaGraphExecDestroy(gexec);
    for (auto& g : gcache) cudaGraphExecDestroy(g.second);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (side.stream) cudaStreamDestroy(side.stream);
    if (side.fork) cudaEventDestroy(side.fork);
    if (side.join) cudaEventDestroy(side.join);
    for (int g = 0; g < sag::kMaxFftGroups; ++g) {
      if (groups.s[g].stream) cudaStreamDestroy(groups.s[g].stream);
      if (groups.s[g].join) cudaEventDestroy(groups.s[g].join);
    }
    for (void* q : allocs) cudaFree(q);
    if (stage_diag) cudaFree(stage_diag);
    if (vjp_pool) cudaFree(vjp_pool);
    if (stage_g) cudaFree(stage_g);
  }
};

namespace sag {
sag_status validate_systems(const sag_system* sys, int32_t B, const sag_options& opt);
sag_status build_plan(const sag_system* sys, int32_t B, const sag_options& opt, sag_plan_s* pl);
sag_status update_factors(sag_plan_s* pl, const double* factors, int on_device);
// Stream groups of the FFT stage (1..4; 1 = one launch per kernel) and the
// plan-time search over them.
sag_status configure_fft_groups(sag_plan_s* pl, int G);
sag_status autotune_fft_groups(sag_plan_s* pl);
// Plan-time search over the four-step split of each order (sag_options.autotune):
// may replace *pl by a plan built with other splits.
sag_status autotune_geometry(const sag_system* sys, int32_t B, const sag_options& opt, sag_plan_s** pl);
}  // namespace sag
