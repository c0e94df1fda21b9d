// C ABI of the library (include/sag.h): error reporting, host-buffer staging,
// the RK2 integrator (stages and CUDA-graph replay), profiling and work
// accounting. Plan construction is in plan_build.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "dw_pow.cuh"
#include "plan_host.h"

using namespace sag;

namespace {
thread_local std::string g_err;
}  // namespace

namespace sag {

sag_status fail(sag_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
sag_status cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return SAG_ECUDA;
}
// Lets other translation units of the library report through sag_last_error.
sag_status set_last_error(sag_status s, const char* msg) {
  g_err = msg;
  return s;
}

void EventHook::mark(int id, cudaStream_t st) {
  if (marks.size() == pool.size()) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) {
      failed = true;
      return;
    }
    pool.push_back(ev);
  }
  cudaEvent_t ev = pool[marks.size()];
  if (cudaEventRecord(ev, st) != cudaSuccess) failed = true;
  marks.emplace_back(id, ev);
}
EventHook::~EventHook() {
  for (cudaEvent_t ev : pool) cudaEventDestroy(ev);
}

}  // namespace sag

namespace {

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

sag_status eval(sag_plan_t pl, const double* nin, EpiArgs A, cudaStream_t st, bool allow_hook = true) {
  A.part = pl->epi_part;
  cudaError_t e = enqueue_eval(pl->P, pl->L, nin, A, st, (pl->prof && allow_hook) ? &pl->hook : nullptr,
                               &pl->side, &pl->groups);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return SAG_OK;
}

// The two stages of one explicit RK2 step (Heun or midpoint) on device state n.
// Runs the work `enqueue` puts on a stream as a CUDA graph: captured once per
// key on the plan's capture stream, then replayed on st.
template <class F>
sag_status replay(sag_plan_t pl, const sag_plan_s::GraphKey& k, cudaStream_t st, F enqueue) {
  cudaGraphExec_t x = nullptr;
  for (auto& it : pl->gcache)
    if (it.first.kind == k.kind && it.first.p0 == k.p0 && it.first.p1 == k.p1 && it.first.dt == k.dt &&
        it.first.p2 == k.p2 && it.first.i0 == k.i0)
      x = it.second;
  cudaError_t e;
  if (!x) {
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_fail(e, "begin capture");
    sag_status s = enqueue(pl->cap_stream);
    e = cudaStreamEndCapture(pl->cap_stream, &g);
    if (s != SAG_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    if (pl->gcache.size() >= 8) {
      cudaGraphExecDestroy(pl->gcache.front().second);
      pl->gcache.erase(pl->gcache.begin());
    }
    pl->gcache.push_back({k, x});
  }
  if ((e = cudaGraphLaunch(x, st)) != cudaSuccess) return cuda_fail(e, "graph launch");
  return SAG_OK;
}

sag_status enqueue_step(sag_plan_t pl, double* n, double dt, double* diag, cudaStream_t st,
                        bool allow_hook, double* nstar = nullptr) {
  // n* = the first stage's state: the plan's buffer, or the caller's (the
  // adjoint keeps the stage states of a recomputed segment)
  double* ns = nstar ? nstar : pl->nstar;
  EpiArgs a{};
  a.nin = n;
  a.k1buf = pl->k1buf;
  a.out0 = ns;
  a.dt = dt;
  a.mode = pl->rk == SAG_HEUN ? EPI_HEUN1 : EPI_MID1;
  a.flux = diag != nullptr;  // the outflow is only reported through diag
  // The first stage writes n*'s double-word copy at n's scale, so the second
  // evaluation starts at its FFTs (the scale is renewed every step).
  a.split_next = pl->P.dwpath;
  sag_status s = eval(pl, n, a, st, allow_hook);
  if (s != SAG_OK) return s;
  EpiArgs b{};
  b.nin = ns;
  b.nbase = n;
  b.k1buf = pl->k1buf;
  b.diag = diag;
  b.dt = dt;
  b.mode = pl->rk == SAG_HEUN ? EPI_HEUN2 : EPI_MID2;
  b.flux = a.flux;
  b.presplit = pl->P.dwpath;
  return eval(pl, ns, b, st, allow_hook);
}

// Operation counts of the double-word arithmetic (FP32 instructions), as
// written in dw.cuh (results left unnormalised): dw_add 8, dw_mul 4, one
// component of a complex product (dot2) 16, so a complex add 16, a complex
// product 32, a real double-word constant times a complex 8, a power-of-two
// scale 4. FP64 arithmetic: a
// complex add 2, a complex product 4 (2 multiplies, 2 FMAs), a real times a
// complex 2.
// The double-word FFT butterflies of radix 2, 3, 4 and 8 run in the
// grid-aligned arithmetic of fft_aligned.cuh instead (grid = true): rounding
// an input's high words to the grid 8 per complex value, a twiddle product
// rounded to the grid 24, a complex add 4, a real constant product 5; the
// radix-2/3/4/8 DFTs then cost 8, 38, 32 and 124 (max-abs and exponent
// operations not counted).
struct OpCost {
  double cadd, cmul, kmul, scale;
  bool grid;
};
constexpr OpCost kCostDW{16, 32, 8, 4, true};
constexpr OpCost kCostDWX{16, 32, 8, 4, false};  // SAG_FP32_SPLIT_EXACT: plain double-word butterflies
constexpr OpCost kCostF64{2, 4, 2, 2, false};

double dft_ops(int R, const OpCost& c) {
  switch (R) {
    case 2: return 2 * c.cadd;
    case 3: return 6 * c.cadd + c.kmul + c.scale;
    case 4: return 8 * c.cadd;
    case 5: return 16 * c.cadd + 8 * c.kmul;
    case 6: return 2 * (6 * c.cadd + c.kmul + c.scale) + 6 * c.cadd;  // two 3-point DFTs, 6 adds
    default: return 26 * c.cadd + 2 * c.kmul;  // radix 8: 8 + 2 + 16 adds, 2 constant products
  }
}

// One length-P transform with the given radix schedule: the compile-time
// schedule of fft_ct.cuh (ct_plan) for the lengths the kernels specialise,
// else the runtime one.
double bfly_ops(int R, bool twiddled, const OpCost& c) {
  if (c.grid && R != 5) {
    const double dft = R == 2 ? 8 : R == 3 ? 38 : R == 4 ? 32 : R == 6 ? 100 : 124;
    return 8 + (R - 1) * (twiddled ? 24 : 8) + dft;
  }
  return dft_ops(R, c) + (twiddled ? (R - 1) * c.cmul : 0.0);
}

radix_plan ct_plan(int P, bool ct, const radix_plan& rt) {
  if (!ct) return rt;
  const ct_sched sc = make_ct_sched(P);
  radix_plan rp{};
  rp.n = sc.n;
  for (int s = 0; s < sc.n; ++s) rp.r[s] = sc.r[s];
  return rp;
}

double fft_ops(int P, const radix_plan& rp, const OpCost& c) {
  double ops = 0.0;
  int Ns = 1;
  for (int s = 0; s < rp.n; ++s) {
    const int R = rp.r[s];
    ops += (double)(P / R) * bfly_ops(R, Ns > 1, c);
    Ns *= R;
  }
  return ops;
}

// SAG_CP_POWER systems as CP systems: every vector U^(m)_r(i) = u pow(i, a)
// (FP64, host libm), in the CP layout, plus the (u, a) list in vector order
// (orders of rank 0 contribute neither).
sag_status expand_power(const sag_system* sys, int32_t B, std::vector<sag_system>* cp,
                        std::vector<std::vector<double>>* store, std::vector<double>* ua) {
  cp->assign(sys, sys + B);
  store->resize(B);
  ua->clear();
  for (int b = 0; b < B; ++b) {
    const sag_system& s = sys[b];
    const std::string at = B > 1 ? " (system " + std::to_string(b) + ")" : "";
    if (s.fmt != SAG_CP_POWER) return fail(SAG_EUNSUPPORTED, "all systems of a plan must share one format" + at);
    if (!s.rank || !s.factors) return fail(SAG_EINVAL, "NULL rank or factors" + at);
    if (s.N < 1 || s.N > (1 << 22) || s.D < 2 || s.D > kMaxD) return fail(SAG_EINVAL, "N in [1, 2^22] and D in [2, 8] required" + at);
    int64_t npar = 0;
    for (int d = 2; d <= s.D; ++d) {
      if (s.rank[d - 2] < 0 || s.rank[d - 2] > 4096) return fail(SAG_EINVAL, "CP rank out of [0, 4096]" + at);
      npar += 2LL * d * s.rank[d - 2];
    }
    std::vector<double> par((size_t)std::max<int64_t>(npar, 1));
    cudaError_t e = cudaMemcpy(par.data(), s.factors, (size_t)npar * sizeof(double),
                               s.factors_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
    if (e != cudaSuccess) return cuda_fail(e, "copy power parameters");
    std::vector<double>& U = (*store)[b];
    U.clear();
    U.reserve((size_t)(npar / 2) * s.N);
    for (int64_t v = 0; v < npar / 2; ++v) {
      const double u = par[2 * v], a = par[2 * v + 1];
      if (!std::isfinite(u) || !std::isfinite(a) || std::fabs(a) > 2.5)
        return fail(SAG_EINVAL, "power factors need finite u and |a| <= 2.5" + at);
      ua->push_back(u);
      ua->push_back(a);
      for (int i = 1; i <= s.N; ++i) U.push_back(u * std::pow((double)i, a));
    }
    (*cp)[b].fmt = SAG_CP;
    (*cp)[b].factors = U.data();
    (*cp)[b].factors_on_device = 0;
  }
  return SAG_OK;
}

}  // namespace

extern "C" {

void sag_default_options(sag_options* opt) {
  if (!opt) return;
  opt->prec = SAG_FP32_SPLIT;
  opt->rk = SAG_HEUN;
  opt->symmetrize_q = 1;
  opt->autotune = 0;
  opt->max_m2 = 0;
  opt->m2 = nullptr;
  opt->n_m2 = 0;
  opt->keep_repeats = 0;
}

const char* sag_last_error(void) { return g_err.c_str(); }

const char* sag_version(void) { return "sag 0.2 (sm_103a)"; }

sag_status sag_plan(const sag_system* sys, int32_t B, const sag_options* opt, sag_plan_t* out) {
  g_err.clear();
  if (!out) return fail(SAG_EINVAL, "out is NULL");
  *out = nullptr;
  sag_options o;
  sag_default_options(&o);
  if (opt) o = *opt;
  // Parametric factors: the plan is built from the expanded CP factors (FP64,
  // u pow(i, a) on the host) and keeps (u, a) for the kernels that generate U.
  std::vector<sag_system> cp;
  std::vector<std::vector<double>> store;
  std::vector<double> ua;
  const sag_system* use = sys;
  if (sys && B >= 1 && B <= 65535 && sys[0].fmt == SAG_CP_POWER) {
    sag_status se = expand_power(sys, B, &cp, &store, &ua);
    if (se != SAG_OK) return se;
    use = cp.data();
  }
  sag_status s = validate_systems(use, B, o);
  if (s != SAG_OK) return s;
  sag_plan_s* pl = new (std::nothrow) sag_plan_s();
  if (!pl) return fail(SAG_ENOMEM, "host allocation");
  pl->pow_ua = std::move(ua);
  s = build_plan(use, B, o, pl);
  if (s == SAG_OK && o.autotune) s = autotune_geometry(use, B, o, &pl);
  if (s != SAG_OK) {
    delete pl;
    return s;
  }
  *out = pl;
  return SAG_OK;
}

sag_status sag_plan_layout(sag_plan_t pl, int64_t* offsets) {
  if (!pl || !offsets) return fail(SAG_EINVAL, "NULL argument");
  for (int b = 0; b <= pl->B; ++b) offsets[b] = pl->offsets[b];
  return SAG_OK;
}

sag_status sag_plan_bytes(sag_plan_t pl, size_t* bytes) {
  if (!pl || !bytes) return fail(SAG_EINVAL, "NULL argument");
  *bytes = pl->bytes;
  return SAG_OK;
}

sag_status sag_rhs_parts(sag_plan_t pl, const double* n, double* p, double* q, double* outflow,
                         void* stream) {
  if (!pl || !n) return fail(SAG_EINVAL, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nb = (size_t)pl->Ntot * sizeof(double);
  const double* nd = n;
  cudaError_t e;
  if (!is_device_ptr(n)) {
    if ((e = cudaMemcpyAsync(pl->stage_a, n, nb, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_fail(e, "copy n");
    nd = pl->stage_a;
  }
  const bool ph = p && !is_device_ptr(p), qh = q && !is_device_ptr(q);
  const bool oh = outflow && !is_device_ptr(outflow);
  EpiArgs a{};
  a.mode = EPI_RHS;
  a.nin = nd;
  a.pout = ph ? pl->stage_b : p;
  a.qout = qh ? pl->stage_c : q;
  a.outflow_out = outflow ? (oh ? pl->dev_outflow : outflow) : nullptr;
  a.flux = outflow != nullptr;
  sag_status s = eval(pl, nd, a, st);
  if (s != SAG_OK) return s;
  if (ph && (e = cudaMemcpyAsync(p, pl->stage_b, nb, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "copy p");
  if (qh && (e = cudaMemcpyAsync(q, pl->stage_c, nb, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "copy q");
  if (oh && (e = cudaMemcpyAsync(outflow, pl->dev_outflow, sizeof(double) * pl->B,
                                 cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "copy outflow");
  if (ph || qh || oh) {
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "sync");
  }
  return SAG_OK;
}

sag_status sag_rhs(sag_plan_t pl, const double* n, double* dndt, void* stream) {
  if (!pl || !n || !dndt) return fail(SAG_EINVAL, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nb = (size_t)pl->Ntot * sizeof(double);
  const double* nd = n;
  cudaError_t e;
  if (!is_device_ptr(n)) {
    if ((e = cudaMemcpyAsync(pl->stage_a, n, nb, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_fail(e, "copy n");
    nd = pl->stage_a;
  }
  const bool oh = !is_device_ptr(dndt);
  EpiArgs a{};
  a.mode = EPI_RHS;
  a.nin = nd;
  a.out0 = oh ? pl->stage_b : dndt;
  // per-kernel profiling launches kernel by kernel; otherwise a cached graph
  sag_status s = pl->prof ? eval(pl, nd, a, st)
                          : replay(pl, {1, nd, a.out0, 0.0}, st,
                                   [&](cudaStream_t cs) { return eval(pl, nd, a, cs, false); });
  if (s != SAG_OK) return s;
  if (oh) {
    if ((e = cudaMemcpyAsync(dndt, pl->stage_b, nb, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "copy dndt");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "sync");
  }
  return SAG_OK;
}

sag_status sag_rk2_step(sag_plan_t pl, double* n, double dt, void* stream) {
  if (!pl || !n) return fail(SAG_EINVAL, "NULL argument");
  if (!std::isfinite(dt)) return fail(SAG_EINVAL, "dt is not finite");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nb = (size_t)pl->Ntot * sizeof(double);
  const bool h = !is_device_ptr(n);
  double* nd = n;
  cudaError_t e;
  if (h) {
    if ((e = cudaMemcpyAsync(pl->stage_a, n, nb, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_fail(e, "copy n");
    nd = pl->stage_a;
  }
  sag_status s = pl->prof ? enqueue_step(pl, nd, dt, nullptr, st, true)
                          : replay(pl, {2, nd, nullptr, dt}, st, [&](cudaStream_t cs) {
                              return enqueue_step(pl, nd, dt, nullptr, cs, false);
                            });
  if (s != SAG_OK) return s;
  if (h) {
    if ((e = cudaMemcpyAsync(n, pl->stage_a, nb, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "copy n back");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "sync");
  }
  return SAG_OK;
}

sag_status sag_power_eval(double u, double a, int32_t N, double* out, void* stream) {
  if (!out) return fail(SAG_EINVAL, "NULL argument");
  if (N < 1 || N > (1 << 22)) return fail(SAG_EINVAL, "N must be in [1, 2^22]");
  if (!std::isfinite(u) || !std::isfinite(a) || std::fabs(a) > 2.5)
    return fail(SAG_EINVAL, "finite u and |a| <= 2.5 required");
  if (!is_device_ptr(out)) return fail(SAG_EINVAL, "out must be a device pointer");
  std::vector<float2> lt((size_t)N + 1, make_float2(0.f, 0.f));
  for (int i = 1; i <= N; ++i) {
    const long double l = logl((long double)i);
    const float hi = (float)l;
    lt[i] = make_float2(hi, (float)(l - hi));
  }
  std::vector<float> ek(kExpConsts);
  make_exp_consts(ek.data());
  const dw ud = dw_from_double(u), ad = dw_from_double(a);
  float2* dlt = nullptr;
  float* dek = nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMalloc(&dlt, lt.size() * sizeof(float2));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc ln table");
  if ((e = cudaMalloc(&dek, ek.size() * sizeof(float))) != cudaSuccess) {
    cudaFree(dlt);
    return cuda_fail(e, "cudaMalloc exp table");
  }
  if ((e = cudaMemcpyAsync(dlt, lt.data(), lt.size() * sizeof(float2), cudaMemcpyHostToDevice, st)) == cudaSuccess &&
      (e = cudaMemcpyAsync(dek, ek.data(), ek.size() * sizeof(float), cudaMemcpyHostToDevice, st)) == cudaSuccess &&
      (e = enqueue_power_eval(make_float4(ud.hi, ud.lo, ad.hi, ad.lo), dlt, dek, N, out, st)) == cudaSuccess)
    e = cudaStreamSynchronize(st);
  cudaFree(dlt);
  cudaFree(dek);
  if (e != cudaSuccess) return cuda_fail(e, "power evaluation");
  return SAG_OK;
}

sag_status sag_rk2_stage(sag_plan_t pl, int32_t stage, double* n, double* nstar, double* k1, const double* k,
                         double dt, void* stream) {
  if (!pl || !n || !nstar || !k1 || !k) return fail(SAG_EINVAL, "NULL argument");
  if (stage != 0 && stage != 1) return fail(SAG_EINVAL, "stage must be 0 or 1");
  if (!std::isfinite(dt)) return fail(SAG_EINVAL, "dt is not finite");
  if (!is_device_ptr(n) || !is_device_ptr(nstar) || !is_device_ptr(k1) || !is_device_ptr(k))
    return fail(SAG_EINVAL, "sag_rk2_stage takes device vectors");
  cudaError_t e = enqueue_rk2_stage(pl->P, stage, pl->rk == SAG_MIDPOINT ? 1 : 0, n, nstar, k1, k, dt,
                                    static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return SAG_OK;
}

sag_status sag_integrate(sag_plan_t pl, double* n, double dt, int64_t steps, double* diag,
                         void* stream) {
  if (!pl || !n) return fail(SAG_EINVAL, "NULL argument");
  if (steps < 0) return fail(SAG_EINVAL, "steps must be >= 0");
  if (!std::isfinite(dt)) return fail(SAG_EINVAL, "dt is not finite");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nb = (size_t)pl->Ntot * sizeof(double);
  const bool nh = !is_device_ptr(n);
  const bool dh = diag && !is_device_ptr(diag);
  double* nd = n;
  double* dd = diag;
  cudaError_t e;
  if (nh) {
    if ((e = cudaMemcpyAsync(pl->stage_a, n, nb, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_fail(e, "copy n");
    nd = pl->stage_a;
  }
  const size_t dlen = (size_t)(steps + 1) * pl->B * 3;
  if (dh) {
    if (pl->stage_diag_len < dlen) {
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "sync");
      if (pl->stage_diag) cudaFree(pl->stage_diag);
      pl->stage_diag = nullptr;
      pl->stage_diag_len = 0;
      if (cudaMalloc(&pl->stage_diag, dlen * sizeof(double)) != cudaSuccess)
        return fail(SAG_ENOMEM, "cudaMalloc diag staging");
      pl->stage_diag_len = dlen;
    }
    dd = pl->stage_diag;
  }
  if ((e = enqueue_moments(pl->P, nd, dd, st)) != cudaSuccess) return cuda_fail(e, "moments");
  if (steps > 0) {
    if (!pl->gexec || pl->g_n != nd || pl->g_dt != dt || pl->g_diag != dd) {
      if (pl->gexec) {
        cudaGraphExecDestroy(pl->gexec);
        pl->gexec = nullptr;
      }
      cudaGraph_t g = nullptr;
      if ((e = cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "begin capture");
      sag_status s = enqueue_step(pl, nd, dt, dd, pl->cap_stream, false);
      e = cudaStreamEndCapture(pl->cap_stream, &g);
      if (s != SAG_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (e != cudaSuccess) return cuda_fail(e, "end capture");
      e = cudaGraphInstantiate(&pl->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
      pl->g_n = nd;
      pl->g_dt = dt;
      pl->g_diag = dd;
    }
    for (int64_t i = 0; i < steps; ++i)
      if ((e = cudaGraphLaunch(pl->gexec, st)) != cudaSuccess) return cuda_fail(e, "graph launch");
  }
  if (nh && (e = cudaMemcpyAsync(n, nd, nb, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "copy n back");
  if (dh && (e = cudaMemcpyAsync(diag, dd, dlen * sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "copy diag back");
  if (nh || dh) {
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "sync");
  }
  return SAG_OK;
}

}  // extern "C"

namespace {

// Checks that the plan can run the vector-Jacobian product.
sag_status vjp_supported(sag_plan_t pl) {
  if (pl->fmt == SAG_TT) {
    if ((int)pl->L.rowtt_smem > smem_limit() || (int)pl->L.vcol_smem > smem_limit())
      return fail(SAG_EUNSUPPORTED, "adjoint blocks exceed shared memory (row or column length too large)");
    return SAG_OK;
  }
  if ((int)pl->L.vrow_smem > smem_limit() || (int)pl->L.vcol_smem > smem_limit())
    return fail(SAG_EUNSUPPORTED, "adjoint row blocks exceed shared memory (order or row length too large)");
  return SAG_OK;
}

// Device view of a caller buffer of `count` doubles: the buffer itself if it
// is device memory, else a plan staging buffer (copied in when `in`).
sag_status stage(sag_plan_t pl, double* user, size_t count, bool in, double** dev, double** pool,
                 size_t* pool_len, cudaStream_t st) {
  if (!user || is_device_ptr(user)) {
    *dev = user;
    return SAG_OK;
  }
  if (*pool_len < count) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "sync");
    if (*pool) cudaFree(*pool);
    *pool = nullptr;
    *pool_len = 0;
    if (cudaMalloc(pool, count * sizeof(double)) != cudaSuccess) return fail(SAG_ENOMEM, "cudaMalloc staging");
    *pool_len = count;
  }
  *dev = *pool;
  if (in) {
    cudaError_t e = cudaMemcpyAsync(*pool, user, count * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy in");
  }
  return SAG_OK;
}

}  // namespace

extern "C" {

sag_status sag_rhs_vjp(sag_plan_t pl, const double* n, const double* g, double* gn, double* gU,
                       void* stream) {
  if (!pl || !n || !g) return fail(SAG_EINVAL, "NULL argument");
  sag_status s = vjp_supported(pl);
  if (s != SAG_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t Nt = (size_t)pl->Ntot;
  double *nd, *gd, *gnd, *gud;
  // n -> stage_a, g -> stage_b, gn -> stage_c (state-sized); gU -> stage_g (factor-sized)
  size_t la = Nt, lb = Nt, lc = Nt;
  if ((s = stage(pl, const_cast<double*>(n), Nt, true, &nd, &pl->stage_a, &la, st)) != SAG_OK ||
      (s = stage(pl, const_cast<double*>(g), Nt, true, &gd, &pl->stage_b, &lb, st)) != SAG_OK ||
      (s = stage(pl, gn, Nt, false, &gnd, &pl->stage_c, &lc, st)) != SAG_OK ||
      (s = stage(pl, gU, (size_t)pl->nfactor, false, &gud, &pl->stage_g, &pl->stage_g_len, st)) != SAG_OK)
    return s;
  cudaError_t e = enqueue_vjp(pl->P, pl->L, nd, gd, gnd, gud, 0, st, &pl->side);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  bool sync = false;
  if (gn && gnd != gn) {
    if ((e = cudaMemcpyAsync(gn, gnd, Nt * sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "copy gn");
    sync = true;
  }
  if (gU && gud != gU) {
    if ((e = cudaMemcpyAsync(gU, gud, (size_t)pl->nfactor * sizeof(double), cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      return cuda_fail(e, "copy gU");
    sync = true;
  }
  if (sync && (e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "sync");
  return SAG_OK;
}

sag_status sag_integrate_vjp(sag_plan_t pl, const double* n0, double dt, int64_t steps, int64_t ckpt,
                             const double* g_final, double* g_n0, double* g_U, void* stream) {
  if (!pl || !n0 || !g_final) return fail(SAG_EINVAL, "NULL argument");
  if (steps < 0) return fail(SAG_EINVAL, "steps must be >= 0");
  if (!std::isfinite(dt)) return fail(SAG_EINVAL, "dt is not finite");
  sag_status s = vjp_supported(pl);
  if (s != SAG_OK) return s;
  if (ckpt <= 0) {
    ckpt = 1;
    while (ckpt * ckpt < steps) ++ckpt;
  }
  if (ckpt > steps && steps > 0) ckpt = steps;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t Nt = (size_t)pl->Ntot;
  const int64_t nck = steps > 0 ? (steps + ckpt - 1) / ckpt : 1;
  // pool: checkpoints [nck], segment states [ckpt], x, gbar, gk, gA, gB,
  // the segment's stage states n* [ckpt]
  const size_t need = ((size_t)nck + 2 * (size_t)ckpt + 5) * Nt;
  cudaError_t e;
  if (pl->vjp_pool_len < need) {
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "sync");
    if (pl->vjp_pool) cudaFree(pl->vjp_pool);
    pl->vjp_pool = nullptr;
    pl->vjp_pool_len = 0;
    if (cudaMalloc(&pl->vjp_pool, need * sizeof(double)) != cudaSuccess)
      return fail(SAG_ENOMEM, "cudaMalloc adjoint checkpoints");
    pl->vjp_pool_len = need;
  }
  double* ck = pl->vjp_pool;
  double* seg = ck + (size_t)nck * Nt;
  double* x = seg + (size_t)ckpt * Nt;
  double* gbar = x + Nt;
  double* gk = gbar + Nt;
  double* gA = gk + Nt;
  double* gB = gA + Nt;
  double* stg = gB + Nt;
  const size_t nb = Nt * sizeof(double);
  const cudaMemcpyKind in_kind = is_device_ptr(n0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  double* gud;
  if ((s = stage(pl, g_U, (size_t)pl->nfactor, false, &gud, &pl->stage_g, &pl->stage_g_len, st)) != SAG_OK)
    return s;
  // Each phase of a segment (its forward steps, the recomputation of its
  // states, its reverse steps) runs as one cached CUDA graph: the buffers are
  // the same for every segment of a given length, only the checkpoint copies
  // between phases differ. With per-kernel profiling on, kernels launch
  // directly.
  auto phase = [&](int kind, const void* p, int64_t len, auto&& body) -> sag_status {
    if (pl->prof) return body(st);
    return replay(pl, {kind, p, gud, dt, seg, len * 65536 + ckpt}, st, body);
  };
  // Forward sweep, keeping the state at the start of every segment.
  if ((e = cudaMemcpyAsync(x, n0, nb, in_kind, st)) != cudaSuccess) return cuda_fail(e, "copy n0");
  for (int64_t c = 0; c < nck && steps > 0; ++c) {
    const int64_t len = std::min<int64_t>(ckpt, steps - c * ckpt);
    if ((e = cudaMemcpyAsync(ck + (size_t)c * Nt, x, nb, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return cuda_fail(e, "checkpoint");
    s = phase(3, x, len, [&](cudaStream_t cs) -> sag_status {
      for (int64_t t = 0; t < len; ++t) {
        sag_status r = enqueue_step(pl, x, dt, nullptr, cs, false);
        if (r != SAG_OK) return r;
      }
      return SAG_OK;
    });
    if (s != SAG_OK) return s;
  }
  // Reverse sweep: recompute each segment's states, then step backwards.
  const cudaMemcpyKind g_kind = is_device_ptr(g_final) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if ((e = cudaMemcpyAsync(gbar, g_final, nb, g_kind, st)) != cudaSuccess) return cuda_fail(e, "copy g");
  if (gud && (e = cudaMemsetAsync(gud, 0, (size_t)pl->nfactor * sizeof(double), st)) != cudaSuccess)
    return cuda_fail(e, "zero gU");
  const bool heun = pl->rk == SAG_HEUN;
  const double h1 = heun ? dt : 0.5 * dt;   // n* = n + h1 k1
  const double w1 = heun ? 0.5 * dt : 0.0;  // weight of k1 in the update
  const double w2 = heun ? 0.5 * dt : dt;   // weight of k2 in the update
  for (int64_t c = nck - 1; c >= 0 && steps > 0; --c) {
    const int64_t t0 = c * ckpt, len = std::min<int64_t>(ckpt, steps - t0);
    if ((e = cudaMemcpyAsync(seg, ck + (size_t)c * Nt, nb, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return cuda_fail(e, "restore");
    if (len > 1) {
      s = phase(4, seg, len, [&](cudaStream_t cs) -> sag_status {
        for (int64_t t = 0; t + 1 < len; ++t) {
          double* cur = seg + (size_t)t * Nt;
          double* nxt = cur + Nt;
          cudaError_t r = cudaMemcpyAsync(nxt, cur, nb, cudaMemcpyDeviceToDevice, cs);
          if (r != cudaSuccess) return cuda_fail(r, "recompute");
          sag_status q = enqueue_step(pl, nxt, dt, nullptr, cs, false, stg + (size_t)t * Nt);
          if (q != SAG_OK) return q;
        }
        return SAG_OK;
      });
      if (s != SAG_OK) return s;
    }
    s = phase(5, seg, len, [&](cudaStream_t cs) -> sag_status {
      for (int64_t t = len - 1; t >= 0; --t) {
        double* n = seg + (size_t)t * Nt;
        // n* of this step: kept by the recomputation, except for the
        // segment's last step, which was not recomputed
        const double* ns = stg + (size_t)t * Nt;
        if (t == len - 1) {
          EpiArgs a{};
          a.nin = n;
          a.k1buf = pl->k1buf;
          a.out0 = pl->nstar;
          a.dt = dt;
          a.mode = heun ? EPI_HEUN1 : EPI_MID1;
          sag_status q = eval(pl, n, a, cs, false);
          if (q != SAG_OK) return q;
          ns = pl->nstar;
        }
        cudaError_t r;
        if ((r = enqueue_axpby(gk, w2, gbar, 0.0, nullptr, (int64_t)Nt, cs)) != cudaSuccess ||
            (r = enqueue_vjp(pl->P, pl->L, ns, gk, gA, gud, 1, cs, &pl->side)) != cudaSuccess ||
            (r = enqueue_axpby(gk, w1, gbar, h1, gA, (int64_t)Nt, cs)) != cudaSuccess ||
            (r = enqueue_vjp(pl->P, pl->L, n, gk, gB, gud, 1, cs, &pl->side)) != cudaSuccess ||
            (r = enqueue_axpby(gbar, 1.0, gbar, 1.0, gA, (int64_t)Nt, cs)) != cudaSuccess ||
            (r = enqueue_axpby(gbar, 1.0, gbar, 1.0, gB, (int64_t)Nt, cs)) != cudaSuccess)
          return cuda_fail(r, "adjoint step");
      }
      return SAG_OK;
    });
    if (s != SAG_OK) return s;
  }
  if (g_n0) {
    const cudaMemcpyKind out_kind = is_device_ptr(g_n0) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if ((e = cudaMemcpyAsync(g_n0, gbar, nb, out_kind, st)) != cudaSuccess) return cuda_fail(e, "copy g_n0");
  }
  if (g_U && gud != g_U &&
      (e = cudaMemcpyAsync(g_U, gud, (size_t)pl->nfactor * sizeof(double), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess)
    return cuda_fail(e, "copy g_U");
  if ((g_n0 && !is_device_ptr(g_n0)) || (g_U && gud != g_U)) {
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "sync");
  }
  return SAG_OK;
}

sag_status sag_plan_update_factors(sag_plan_t pl, const double* factors, int32_t on_device) {
  if (!pl || !factors) return fail(SAG_EINVAL, "NULL argument");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  return update_factors(pl, factors, on_device);
}

sag_status sag_plan_factor_count(sag_plan_t pl, int64_t* count) {
  if (!pl || !count) return fail(SAG_EINVAL, "NULL argument");
  *count = pl->nfactor;
  return SAG_OK;
}

sag_status sag_plan_set_wait_limit(sag_plan_t pl, int64_t cycles, int32_t unmet) {
  if (!pl) return fail(SAG_EINVAL, "NULL plan");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  pl->P.spin_limit = cycles > 0 ? (long long)cycles : kDefaultSpinLimit;
  pl->P.wait_unmet = unmet ? 1 : 0;
  // captured graphs hold the old limit in their kernel parameters
  for (auto& g : pl->gcache) cudaGraphExecDestroy(g.second);
  pl->gcache.clear();
  if (pl->gexec) {
    cudaGraphExecDestroy(pl->gexec);
    pl->gexec = nullptr;
  }
  return SAG_OK;
}

sag_status sag_sync_status(sag_plan_t pl, void* stream) {
  if (!pl) return fail(SAG_EINVAL, "NULL plan");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  unsigned int status = 0;
  if ((e = cudaMemcpy(&status, pl->P.status, sizeof(unsigned), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "read status");
  if (status) {
    if ((e = cudaMemset(pl->P.status, 0, sizeof(unsigned))) != cudaSuccess) return cuda_fail(e, "clear status");
    if (status & kStatusTimeoutUndrained)
      return fail(SAG_ETIMEOUT,
                  "a device-side wait timed out and a block exited with bulk copies still in flight: "
                  "treat the CUDA context as suspect");
    if (status & kStatusTimeout) return fail(SAG_ETIMEOUT, "a device-side wait timed out");
    return fail(SAG_ENONFINITE, "the right-hand side produced Inf or NaN");
  }
  return SAG_OK;
}

sag_status sag_profile_enable(sag_plan_t pl, int32_t on) {
  if (!pl) return fail(SAG_EINVAL, "NULL plan");
  pl->prof = on != 0;
  return SAG_OK;
}

sag_status sag_profile_read(sag_plan_t pl, double* ms, int64_t* launches, int32_t n) {
  if (!pl || (n > 0 && (!ms || !launches))) return fail(SAG_EINVAL, "NULL argument");
  EventHook& h = pl->hook;
  if (h.failed) {
    h.marks.clear();
    h.failed = false;
    return fail(SAG_ECUDA, "event record failed while profiling");
  }
  if (!h.marks.empty()) {
    cudaError_t e = cudaEventSynchronize(h.marks.back().second);
    if (e != cudaSuccess) return cuda_fail(e, "event sync");
  }
  for (size_t i = 0; i + 1 < h.marks.size(); ++i) {
    const int id = h.marks[i].first;
    if (id < 0 || id >= n) continue;
    float t = 0.f;
    cudaError_t e = cudaEventElapsedTime(&t, h.marks[i].second, h.marks[i + 1].second);
    if (e != cudaSuccess) return cuda_fail(e, "event elapsed time");
    ms[id] += t;
    launches[id] += 1;
  }
  h.marks.clear();
  return SAG_OK;
}

const char* sag_kernel_name(int32_t id) {
  static const char* names[KID_COUNT] = {"k_nmax",    "k_nsplit",      "k_dot",       "k_fwd_col",
                                         "k_rows",    "k_inv_col",     "k_epilogue",  "k_moments",
                                         "k_coef",    "k_rows_tt_fwd", "k_tt_chain",  "k_rows_tt_inv",
                                         "k_qterm"};
  return (id >= 0 && id < KID_COUNT) ? names[id] : nullptr;
}

sag_status sag_kernel_work(sag_plan_t pl, int32_t id, double* ops, int32_t* ops_fp64, double* bytes) {
  if (!pl || !ops || !ops_fp64 || !bytes) return fail(SAG_EINVAL, "NULL argument");
  if (id < 0 || id >= KID_COUNT) return fail(SAG_EINVAL, "kernel id out of range");
  const bool dwp = pl->P.dwpath != 0;
  const OpCost& c = dwp ? (pl->P.exact ? kCostDWX : kCostDW) : kCostF64;
  const double Nt = (double)pl->Ntot, V = pl->P.Vtot;
  const double load_mul = dwp ? 4.0 : 1.0;  // a = U n: dw_mul or one FP64 multiply
  double o = 0.0, b = 0.0;
  int fp64 = dwp ? 0 : 1;
  double factor_elems = 0.0, distinct_elems = 0.0;  // sum over vectors (distinct vectors) of their length
  for (const SysDesc& s : pl->systems) {
    factor_elems += (double)(s.vend - s.vbeg) * s.N;
    distinct_elems += (double)(s.dend - s.dbeg) * s.N;
  }
  switch (id) {
    case KID_NMAX:
      o = 2 * Nt;
      b = 8 * Nt;
      fp64 = 1;
      break;
    case KID_NSPLIT:
      o = 4 * Nt;
      b = 16 * Nt;
      fp64 = 1;
      break;
    case KID_DOT:  // one FP64 FMA (acc += u n) per factor element; the outflow's t = <k U, n>
                   // adds a second only when it is asked for (not counted here)
      o = distinct_elems;  // repeated vectors: once per set
      b = 8 * distinct_elems + 8 * Nt;
      fp64 = 1;
      break;
    case KID_COEF:
      o = 4 * V;
      b = 16 * V * pl->P.maxdotchunk;
      fp64 = 1;
      break;
    case KID_FWD_COL:
      for (const OrderDesc& od : pl->items)  // a pair costs what two single vectors cost
        o += (od.pair ? 2.0 * od.npair : (double)od.nu) *
             (od.M2 * fft_ops(od.M1, ct_plan(od.M1, dwp && od.ct1, od.rp1), c) + (double)od.M * c.cmul + 2.0 * std::min<double>(od.M, od.N) * load_mul);
      b = 8.0 * factor_elems + 8.0 * Nt;
      break;
    case KID_ROWS:
      for (const OrderDesc& od : pl->items) {
        const double Vd = od.nvec, M = od.M;
        const double unpack = 4 * c.cadd + c.cmul;
        const double repack = 4 * c.cadd + c.cmul;
        if (od.pair)  // rows of 2 M2 points per pair; separation: 2 complex adds per pair and index
          o += (double)od.npair * od.M1 * fft_ops(2 * od.M2, ct_plan(2 * od.M2, true, make_radix_plan(2 * od.M2)), c) +
               (double)od.npair * M * 2 * c.cadd;
        else {  // forward rows of every vector; with a slot map (repeated vectors), of each distinct one
          const double Vr = (dwp && od.ct2 && od.umap_off >= 0) ? (double)od.nu : Vd;
          o += Vr * od.M1 * fft_ops(od.M2, ct_plan(od.M2, dwp && od.ct2, od.rp2), c)
               + Vr * M * unpack;                        // real split
        }
        o += (Vd - od.R) * M * c.cmul                           // product over the modes
             + (double)od.R * M * (c.cadd + (dwp ? c.scale : 0))  // rank sum
             + M * repack + od.M1 * fft_ops(od.M2, ct_plan(od.M2, dwp && od.ct2, od.rp2), c)     // inverse rows
             + M * c.cmul;                                        // four-step twiddle
      }
      b = 0.0;  // reads and writes only the FFT workspace
      break;
    case KID_ROWS_TT:
      for (const OrderDesc& od : pl->items)
        o += (double)od.nvec * (od.M1 * fft_ops(od.M2, ct_plan(od.M2, dwp && od.ct2, od.rp2), c) + (double)od.M * (4 * c.cadd + c.cmul));
      break;
    case KID_TT_CHAIN:
      for (const OrderDesc& od : pl->items) o += (double)od.nvec * (od.M + 1) * (c.cmul + c.cadd);
      break;
    case KID_ROWS_TT_INV:
      for (const OrderDesc& od : pl->items)
        o += (double)od.M * (4 * c.cadd + 2 * c.cmul) + od.M1 * fft_ops(od.M2, ct_plan(od.M2, dwp && od.ct2, od.rp2), c);
      break;
    case KID_INV_COL:
      for (const OrderDesc& od : pl->items) o += od.M2 * fft_ops(od.M1, ct_plan(od.M1, dwp && od.ct1, od.rp1), c);
      b = 0.0;
      for (const OrderDesc& od : pl->items) b += 8.0 * od.N;  // P^(d) written
      break;
    case KID_QTERM:  // q = n (sum_v coef_v U_v(k))
      o = distinct_elems + Nt;
      b = 8 * distinct_elems + 2 * 8 * Nt;
      fp64 = 1;
      break;
    case KID_EPILOGUE:  // rhs = p + q; stage update; moments
      o = 8 * Nt;
      b = 8.0 * pl->items.size() / std::max(1, pl->B) * Nt + 4 * 8 * Nt;
      fp64 = 1;
      break;
    case KID_MOMENTS:
      o = 3 * Nt;
      b = 8 * Nt;
      fp64 = 1;
      break;
  }
  *ops = o;
  *ops_fp64 = fp64;
  *bytes = b;
  return SAG_OK;
}

sag_status sag_kernel_method_work(sag_plan_t pl, int32_t id, double* flops, double* workspace_bytes) {
  if (!pl || !flops || !workspace_bytes) return fail(SAG_EINVAL, "NULL argument");
  if (id < 0 || id >= KID_COUNT) return fail(SAG_EINVAL, "kernel id out of range");
  // Nominal flops of the method (Sec. 1: d-fold convolutions by FFT, inner
  // products), independent of the arithmetic that carries them out: a real
  // FFT of length L is 2.5 L log2 L flops, split between the four-step
  // halves as 2.5 L log2 M1 (columns) and 2.5 L log2 M2 (rows) with the
  // four-step twiddle products (3 L: L/2 complex products of 6 flops) on the
  // column side; a complex product 6, a complex add 2, an FMA 2.
  // Workspace: each transformed vector's four-step intermediate, M = L/2
  // complex values of 16 bytes (double-word or FP64), written by the forward
  // columns and read by the rows; each order's spectral sum, written by the
  // rows and read by the inverse columns.
  double f = 0.0, w = 0.0;
  double factor_elems = 0.0;
  for (const SysDesc& s : pl->systems) factor_elems += (double)(s.vend - s.vbeg) * s.N;
  const double Nt = (double)pl->Ntot;
  for (const OrderDesc& od : pl->items) {
    const double L = od.L, M = od.M, nu = od.pair ? 2.0 * od.npair : (double)od.nu;
    const double lg1 = std::log2((double)od.M1), lg2 = std::log2((double)od.M2);
    switch (id) {
      case KID_FWD_COL:
        f += nu * (od.N + 2.5 * L * lg1 + 3.0 * L);
        w += nu * 16.0 * M;
        break;
      case KID_ROWS:
        f += nu * (2.5 * L * lg2 + 5.0 * L)                       // forward rows and the real split
             + (M + 1) * (6.0 * (od.nvec - od.R) + 2.0 * od.R)   // products over the modes, rank sum
             + 2.5 * L * lg2 + 5.0 * L;                           // repack and inverse rows
        w += nu * 16.0 * M + 16.0 * M;
        break;
      case KID_ROWS_TT:
        f += od.nvec * (2.5 * L * lg2 + 5.0 * L);
        w += od.nvec * 16.0 * M * 2.0;
        break;
      case KID_TT_CHAIN:
        f += od.nvec * (M + 1) * 8.0;
        w += od.nvec * 16.0 * M + 16.0 * M;
        break;
      case KID_ROWS_TT_INV:
        f += 2.5 * L * lg2 + 5.0 * L;
        w += 2.0 * 16.0 * M;
        break;
      case KID_INV_COL:
        f += 2.5 * L * lg1 + 3.0 * L;
        w += 16.0 * M;
        break;
      default:
        break;
    }
  }
  switch (id) {
    case KID_NMAX: f = Nt; break;
    case KID_NSPLIT: f = 2 * Nt; break;
    case KID_DOT: f = 2 * factor_elems; break;
    case KID_COEF: f = 4.0 * pl->P.Vtot; break;
    case KID_QTERM: f = 2 * factor_elems + Nt; break;
    case KID_EPILOGUE: f = 8 * Nt; break;
    case KID_MOMENTS: f = 3 * Nt; break;
    default: break;
  }
  *flops = f;
  *workspace_bytes = w;
  return SAG_OK;
}

namespace {

// Kernel launches of one sag_integrate step (no diagnostics): the kernel
// nodes of the step captured as a graph, which is not launched. -1 if the
// capture fails.
int step_kernel_launches(sag_plan_t pl) {
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return -1;
  const sag_status s = enqueue_step(pl, pl->stage_a, 0.0, nullptr, pl->cap_stream, false);
  const cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &g);
  int count = -1;
  size_t nn = 0;
  if (s == SAG_OK && e == cudaSuccess && g && cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess) {
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess) {
      count = 0;
      for (cudaGraphNode_t x : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(x, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++count;
      }
    }
  }
  if (g) cudaGraphDestroy(g);
  return count;
}

}  // namespace

sag_status sag_plan_describe(sag_plan_t pl, char* buf, size_t len) {
  if (!pl || !buf || len == 0) return fail(SAG_EINVAL, "NULL argument");
  const RhsParams& P = pl->P;
  auto rps = [](const radix_plan& rp) {
    std::string r = "[";
    for (int s = 0; s < rp.n; ++s) r += (s ? ", " : "") + std::to_string(rp.r[s]);
    return r + "]";
  };
  std::string js = "{\"B\": " + std::to_string(P.B) + ", \"Ntot\": " + std::to_string(pl->Ntot) +
                   ", \"format\": \"" + (pl->fmt == SAG_TT ? "tt" : "cp") + "\", \"precision\": \"" +
                   (P.dwpath ? (P.exact ? "fp32_split_exact" : "fp32_split") : "fp64") + "\", \"vectors\": " + std::to_string(P.Vtot) +
                   ", \"orders\": [";
  const size_t shown = std::min<size_t>(pl->items.size(), 16);
  for (size_t i = 0; i < shown; ++i) {
    const OrderDesc& od = pl->items[i];
    js += std::string(i ? ", " : "") + "{\"sys\": " + std::to_string(od.sys) + ", \"d\": " +
          std::to_string(od.d) + ", \"vectors\": " + std::to_string(od.nvec) +
          ", \"transformed\": " + std::to_string(od.pair ? 2 * od.npair : od.nu) +
          ", \"pairs\": " + std::to_string(od.pair) + ", \"parametric\": " + std::to_string(od.pw) +
          ", \"L\": " +
          std::to_string(od.L) + ", \"M1\": " + std::to_string(od.M1) + ", \"M2\": " +
          std::to_string(od.M2) + ", \"radix_M1\": " + rps(od.rp1) + ", \"radix_M2\": " + rps(od.rp2) +
          ", \"W\": " + std::to_string(od.W) + ", \"G\": " + std::to_string(od.G) +
          ", \"compile_time\": [" + std::to_string(od.ct1) + ", " + std::to_string(od.ct2 || od.ctt) + "]}";
  }
  js += "], \"orders_total\": " + std::to_string(pl->items.size()) + ", \"blocks\": {\"fwd_col\": " +
        std::to_string(pl->L.col_blocks) + ", \"rows\": " + std::to_string(pl->L.row_blocks) +
        ", \"fft_groups\": " + std::to_string(pl->fft_groups) +
        ", \"inv_col\": " + std::to_string(pl->L.inv_blocks) + ", \"epilogue\": " +
        std::to_string(pl->L.epi_blocks) + "}, \"device_bytes\": " + std::to_string(pl->bytes) +
        ", \"launches_per_step\": " + std::to_string(step_kernel_launches(pl)) +
        ", \"geometry_autotune\": [" + pl->tune_log + "]}";
  std::snprintf(buf, len, "%s", js.c_str());
  return SAG_OK;
}

void sag_plan_destroy(sag_plan_t pl) {
  if (!pl) return;
  cudaDeviceSynchronize();
  delete pl;
}

}  // extern "C"
