// C ABI of the library (include/sag.h): validation, plan construction
// (FFT geometry, twiddle tables, factor copies, workspace), and the host side
// of sag_rhs / sag_rk2_step / sag_integrate.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "launch.h"
#include "sag.h"

using namespace sag;

namespace {

thread_local std::string g_err;

sag_status fail(sag_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
sag_status cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return SAG_ECUDA;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

double factorial(int d) {
  double f = 1.0;
  for (int i = 2; i <= d; ++i) f *= i;
  return f;
}

// Smallest L = 2^a f (f in {1, 3, 5, 15}, a >= 1) with L >= need.
int64_t choose_fft_length(int64_t need) {
  int64_t best = -1;
  const int64_t fs[4] = {1, 3, 5, 15};
  for (int64_t f : fs) {
    int64_t L = 2 * f;
    while (L < need) L *= 2;
    if (best < 0 || L < best) best = L;
  }
  return best;
}

// omega_P^k = exp(-2 pi i k / P) in FP64.
void unit_root(int64_t k, int64_t P, double& c, double& s) {
  const double a = 2.0 * M_PI * (double)(k % P) / (double)P;
  c = std::cos(a);
  s = -std::sin(a);
}

}  // namespace

namespace sag {
// Lets other translation units of the library report through sag_last_error.
sag_status set_last_error(sag_status s, const char* msg) {
  g_err = msg;
  return s;
}
}  // namespace sag

// Records one CUDA event before each kernel launch and one after the last.
struct EventHook : LaunchHook {
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, cudaEvent_t>> marks;
  bool failed = false;
  void mark(int id, cudaStream_t st) override {
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
  ~EventHook() override {
    for (cudaEvent_t ev : pool) cudaEventDestroy(ev);
  }
};

struct sag_plan_s {
  RhsParams P{};
  LaunchCfg L{};
  int N = 0, D = 0, fmt = 0, prec = 0, rk = 0, sym = 1;
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
  bool prof = false;
  EventHook hook;
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
  ~sag_plan_s() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (void* q : allocs) cudaFree(q);
    if (stage_diag) cudaFree(stage_diag);
  }
};

namespace {

// Twiddles of one order, converted to the path's complex type.
template <class C>
C to_c(double re, double im);
template <>
cd to_c<cd>(double re, double im) { return cd{re, im}; }
template <>
cdw to_c<cdw>(double re, double im) {
  dw r = dw_from_double(re), i = dw_from_double(im);
  return cdw{r.hi, r.lo, i.hi, i.lo};
}

template <class C>
cudaError_t upload_table(sag_plan_s* pl, int64_t P, int64_t count, const void** out) {
  std::vector<C> h(count);
  for (int64_t k = 0; k < count; ++k) {
    double c, s;
    unit_root(k, P, c, s);
    h[k] = to_c<C>(c, s);
  }
  C* d = nullptr;
  cudaError_t e = pl->alloc(&d, count);
  if (e != cudaSuccess) return e;
  *out = d;
  return cudaMemcpy(d, h.data(), count * sizeof(C), cudaMemcpyHostToDevice);
}

template <class C>
cudaError_t upload_order_tables(sag_plan_s* pl, OrderDesc& od) {
  cudaError_t e = upload_table<C>(pl, od.M1, od.M1, &od.tw1);
  if (e == cudaSuccess) e = upload_table<C>(pl, od.M2, od.M2, &od.tw2);
  if (e == cudaSuccess) e = upload_table<C>(pl, od.M, od.M, &od.tw4);
  if (e == cudaSuccess) e = upload_table<C>(pl, od.L, od.M, &od.twL);
  return e;
}

sag_status build_plan(const sag_system* sys, const sag_options& opt, sag_plan_s* pl) {
  const int N = sys->N, D = sys->D;
  pl->N = N;
  pl->D = D;
  pl->fmt = sys->fmt;
  pl->prec = opt.prec;
  pl->rk = opt.rk;
  pl->sym = opt.symmetrize_q;
  const bool dwp = opt.prec == SAG_FP32_SPLIT;
  const size_t csize = dwp ? sizeof(cdw) : sizeof(cd);
  RhsParams& P = pl->P;
  P.N = N;
  P.D = D;
  P.nord = D - 1;
  P.sym = opt.symmetrize_q;
  P.dwpath = dwp ? 1 : 0;

  // Orders: ranks, vector bases, FFT geometry.
  int Vtot = 0;
  int64_t scr = 0, scr2 = 0;
  int colpre = 0, rowpre = 0, invpre = 0;
  size_t col_smem = 0, row_smem = 0;
  for (int d = 2; d <= D; ++d) {
    OrderDesc& od = P.ord[d - 2];
    od.d = d;
    od.R = sys->rank[d - 2];
    od.vbase = Vtot;
    Vtot += d * od.R;
    const int64_t L = choose_fft_length(std::max<int64_t>((int64_t)d * N, 16));
    if (L > (int64_t)1 << 24) return fail(SAG_EUNSUPPORTED, "FFT length above 2^24 (d N too large)");
    od.L = (int)L;
    od.M = (int)(L / 2);
    int M2 = 1;
    while ((int64_t)(2 * M2) * (2 * M2) <= od.M && 2 * M2 <= 512 && od.M % (2 * M2) == 0) M2 *= 2;
    od.M2 = M2;
    od.M1 = od.M / M2;
    if (od.M1 > 4096) return fail(SAG_EUNSUPPORTED, "FFT column length above 4096");
    od.rp1 = make_radix_plan(od.M1);
    od.rp2 = make_radix_plan(od.M2);
    if (od.rp1.n < 0 || od.rp2.n < 0) return fail(SAG_EUNSUPPORTED, "FFT length not a supported product");
    // Compile-time kernels (double-word path) for the common lengths.
    od.ct1 = (dwp && ct_supported(od.M1) && M2 >= ct_cols(od.M1)) ? 1 : 0;
    od.ct2 = (dwp && ct_supported(od.M2) && od.M2 <= 512) ? 1 : 0;
    int W = 1;
    while (2 * W <= M2 && (int64_t)2 * W * od.M1 <= 2048) W *= 2;
    if (od.ct1) W = ct_cols(od.M1);
    od.W = W;
    od.ld1 = od.M1 + 1;
    od.ld2 = od.M2 + 1;
    od.ncolblk = M2 / W;
    od.nrowpair = od.M1 / 2 + 1;
    int G = std::max(1, 2048 / (2 * M2));
    G = std::min(G, d * od.R);
    G = std::min(G, 64);
    if (od.ct2) G = ct_group(od.M2);
    if (dwp && !od.ct2 && 2 * od.M2 > kThreads)
      return fail(SAG_EUNSUPPORTED, "row length without a compile-time kernel above 128");
    od.G = G;
    od.scr_off = scr;
    scr += (int64_t)d * od.R * od.M;
    od.scr2_off = scr2;
    scr2 += od.M;
    P.colpre[d - 2] = colpre;
    P.rowpre[d - 2] = rowpre;
    P.invpre[d - 2] = invpre;
    colpre += d * od.R * od.ncolblk;
    rowpre += od.nrowpair;
    invpre += od.ncolblk;
    // Compile-time kernels work in place (one buffer), the generic ones ping-pong.
    col_smem = std::max(col_smem, (size_t)((od.ct1 ? 1 : 2) * W * od.ld1 + od.M1) * csize);
    // The compile-time row kernel double-buffers its input through bulk copies
    // (two stages plus two mbarriers).
    row_smem = std::max(row_smem, (size_t)(2 * G * 2 * od.ld2 + od.M2) * csize + (od.ct2 ? 16 : 0));
  }
  P.colpre[D - 1] = colpre;
  P.rowpre[D - 1] = rowpre;
  P.invpre[D - 1] = invpre;
  P.Vtot = Vtot;
  P.spin_limit = 4000000000LL;  // about 2 s at the maximum SM clock
  P.dotchunk = 8192;
  P.ndotchunk = (N + P.dotchunk - 1) / P.dotchunk;

  LaunchCfg& L = pl->L;
  L.prep_blocks = std::max(1, std::min(1024, (N + 255) / 256));
  L.col_blocks = colpre;
  L.row_blocks = rowpre;
  L.inv_blocks = invpre;
  L.epi_blocks = (N + 255) / 256;
  L.col_smem = col_smem;
  L.row_smem = row_smem;
  L.inv_smem = col_smem;
  L.epi_smem = (size_t)2 * Vtot * sizeof(double);
  if (col_smem > 227 * 1024 || row_smem > 227 * 1024 || L.epi_smem > 200 * 1024)
    return fail(SAG_EUNSUPPORTED, "shared-memory footprint above the per-block limit");

  // Factors: FP64 copy (inner products, loss term, FP64 FFT input).
  const size_t nf = (size_t)Vtot * N;
  std::vector<double> hf(nf);
  cudaError_t e = cudaMemcpy(hf.data(), sys->factors, nf * sizeof(double),
                             sys->factors_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
  if (e != cudaSuccess) return cuda_fail(e, "copy factors");
  for (size_t i = 0; i < nf; ++i)
    if (!std::isfinite(hf[i])) return fail(SAG_EINVAL, "factors contain Inf or NaN");
  double* U64 = nullptr;
  if ((e = pl->alloc(&U64, nf)) != cudaSuccess) return fail(SAG_ENOMEM, "cudaMalloc factors");
  if ((e = cudaMemcpy(U64, hf.data(), nf * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "upload factors");
  P.U64 = U64;

  // Double-word copy: each vector scaled by 2^-e_v so that max |U| lies in
  // [0.5, 1); the rank term r of order d then carries 2^(sigma_r - E_d) with
  // sigma_r = sum_m e_{v(m,r)}, E_d = max_r sigma_r, and 2^E_d moves into the
  // final FP64 scale of P^(d).
  std::vector<int> ev(Vtot, 0);
  if (dwp) {
    std::vector<float2> hdw(nf);
    for (int v = 0; v < Vtot; ++v) {
      double mx = 0.0;
      for (int k = 0; k < N; ++k) mx = std::max(mx, std::fabs(hf[(size_t)v * N + k]));
      int ex = 0;
      if (mx > 0.0) std::frexp(mx, &ex);
      ev[v] = ex;
      for (int k = 0; k < N; ++k) {
        dw x = dw_from_double(std::ldexp(hf[(size_t)v * N + k], -ex));
        hdw[(size_t)v * N + k] = make_float2(x.hi, x.lo);
      }
    }
    float2* Udw = nullptr;
    if ((e = pl->alloc(&Udw, nf)) != cudaSuccess) return fail(SAG_ENOMEM, "cudaMalloc dw factors");
    if ((e = cudaMemcpy(Udw, hdw.data(), nf * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "upload dw factors");
    P.Udw = Udw;
    float2* ndw = nullptr;
    if ((e = pl->alloc(&ndw, N)) != cudaSuccess) return fail(SAG_ENOMEM, "cudaMalloc n");
    P.ndw = ndw;
  }
  for (int d = 2; d <= D; ++d) {
    OrderDesc& od = P.ord[d - 2];
    int Ed = 0;
    std::vector<float> rs(od.R, 1.0f);
    if (dwp) {
      std::vector<int> sig(od.R, 0);
      for (int r = 0; r < od.R; ++r)
        for (int m = 0; m < d; ++m) sig[r] += ev[od.vbase + m * od.R + r];
      Ed = sig[0];
      for (int r = 1; r < od.R; ++r) Ed = std::max(Ed, sig[r]);
      for (int r = 0; r < od.R; ++r) rs[r] = std::ldexp(1.0f, sig[r] - Ed);
      float* drs = nullptr;
      if ((e = pl->alloc(&drs, od.R)) != cudaSuccess) return fail(SAG_ENOMEM, "cudaMalloc rank scales");
      if ((e = cudaMemcpy(drs, rs.data(), od.R * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "upload rank scales");
      od.rscale = drs;
      e = upload_order_tables<cdw>(pl, od);
    } else {
      od.rscale = nullptr;
      e = upload_order_tables<cd>(pl, od);
    }
    if (e != cudaSuccess) return cuda_fail(e, "twiddle tables");
    // Two factors of 2 per mode come from the real split (2 A[k] per mode),
    // 1/L from the unnormalised inverse, 1/d! from the definition of p^(d).
    od.pscale = std::ldexp(1.0, Ed - d) / ((double)od.L * factorial(d));
  }

  // Workspace.
  void* scratch = nullptr;
  void* scratch2 = nullptr;
  if ((e = pl->alloc((unsigned char**)&scratch, (size_t)scr * csize)) != cudaSuccess ||
      (e = pl->alloc((unsigned char**)&scratch2, (size_t)scr2 * csize)) != cudaSuccess)
    return fail(SAG_ENOMEM, "cudaMalloc FFT workspace");
  P.scratch = scratch;
  P.scratch2 = scratch2;
  if (pl->alloc(&P.pd, (size_t)P.nord * N) != cudaSuccess ||
      pl->alloc(&P.dot_s, (size_t)Vtot * P.ndotchunk) != cudaSuccess ||
      pl->alloc(&P.dot_t, (size_t)Vtot * P.ndotchunk) != cudaSuccess ||
      pl->alloc(&pl->epi_part, (size_t)L.epi_blocks * 4) != cudaSuccess ||
      pl->alloc(&P.sc, 1) != cudaSuccess || pl->alloc(&pl->nstar, N) != cudaSuccess ||
      pl->alloc(&pl->k1buf, N) != cudaSuccess || pl->alloc(&pl->stage_a, N) != cudaSuccess ||
      pl->alloc(&pl->stage_b, N) != cudaSuccess || pl->alloc(&pl->stage_c, N) != cudaSuccess ||
      pl->alloc(&pl->dev_outflow, 1) != cudaSuccess)
    return fail(SAG_ENOMEM, "cudaMalloc workspace");
  P.epi_part = pl->epi_part;
  if ((e = cudaMemset(P.sc, 0, sizeof(DevScalars))) != cudaSuccess) return cuda_fail(e, "memset");

  e = setup_common_kernels(L);
  if (e == cudaSuccess) e = dwp ? setup_fft_kernels_dw(L) : setup_fft_kernels_f64(L);
  if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
  if ((e = cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "stream");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "plan setup");
  return SAG_OK;
}

sag_status validate(const sag_system* sys, int32_t B, const sag_options& opt) {
  if (!sys) return fail(SAG_EINVAL, "sys is NULL");
  if (B < 1) return fail(SAG_EINVAL, "B must be >= 1");
  if (B > 1) return fail(SAG_EUNSUPPORTED, "batched plans (B > 1) are not implemented in this build");
  if (sys->N < 1) return fail(SAG_EINVAL, "N must be >= 1");
  if (sys->D < 2 || sys->D > kMaxD) return fail(SAG_EINVAL, "D must be in [2, 8]");
  if (!sys->rank) return fail(SAG_EINVAL, "rank is NULL");
  if (!sys->factors) return fail(SAG_EINVAL, "factors is NULL");
  if (sys->fmt != SAG_CP && sys->fmt != SAG_TT) return fail(SAG_EINVAL, "unknown format");
  if (sys->fmt == SAG_TT) return fail(SAG_EUNSUPPORTED, "TT kernels are not implemented in this build");
  for (int d = 2; d <= sys->D; ++d)
    if (sys->rank[d - 2] < 1 || sys->rank[d - 2] > 4096) return fail(SAG_EINVAL, "CP rank out of [1, 4096]");
  if (opt.prec != SAG_FP64 && opt.prec != SAG_FP32_SPLIT) return fail(SAG_EINVAL, "unknown precision");
  if (opt.rk != SAG_HEUN && opt.rk != SAG_MIDPOINT) return fail(SAG_EINVAL, "unknown RK2 variant");
  if (opt.symmetrize_q != 0 && opt.symmetrize_q != 1) return fail(SAG_EINVAL, "symmetrize_q must be 0 or 1");
  int64_t nf = 0;
  for (int d = 2; d <= sys->D; ++d) nf += (int64_t)d * sys->rank[d - 2] * sys->N;
  if (nf > ((int64_t)1 << 34)) return fail(SAG_EINVAL, "factor array too large");
  return SAG_OK;
}

// Device-resident views of caller buffers, with host staging.
struct Staged {
  const double* in;
  double* out;
};

sag_status eval(sag_plan_t pl, const double* nin, EpiArgs A, cudaStream_t st, bool allow_hook = true) {
  A.part = pl->epi_part;
  cudaError_t e = enqueue_eval(pl->P, pl->L, nin, A, st, (pl->prof && allow_hook) ? &pl->hook : nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return SAG_OK;
}

sag_status enqueue_step(sag_plan_t pl, double* n, double dt, double* diag, cudaStream_t st,
                        bool allow_hook) {
  EpiArgs a{};
  a.nin = n;
  a.k1buf = pl->k1buf;
  a.out0 = pl->nstar;
  a.dt = dt;
  a.mode = pl->rk == SAG_HEUN ? EPI_HEUN1 : EPI_MID1;
  sag_status s = eval(pl, n, a, st, allow_hook);
  if (s != SAG_OK) return s;
  EpiArgs b{};
  b.nin = pl->nstar;
  b.nbase = n;
  b.k1buf = pl->k1buf;
  b.diag = diag;
  b.dt = dt;
  b.mode = pl->rk == SAG_HEUN ? EPI_HEUN2 : EPI_MID2;
  return eval(pl, pl->nstar, b, st, allow_hook);
}

}  // namespace

extern "C" {

void sag_default_options(sag_options* opt) {
  if (!opt) return;
  opt->prec = SAG_FP32_SPLIT;
  opt->rk = SAG_HEUN;
  opt->symmetrize_q = 1;
  opt->reserved = 0;
}

const char* sag_last_error(void) { return g_err.c_str(); }

const char* sag_version(void) { return "sag 0.1 (sm_103a)"; }

sag_status sag_plan(const sag_system* sys, int32_t B, const sag_options* opt, sag_plan_t* out) {
  g_err.clear();
  if (!out) return fail(SAG_EINVAL, "out is NULL");
  *out = nullptr;
  sag_options o;
  sag_default_options(&o);
  if (opt) o = *opt;
  sag_status s = validate(sys, B, o);
  if (s != SAG_OK) return s;
  sag_plan_s* pl = new (std::nothrow) sag_plan_s();
  if (!pl) return fail(SAG_ENOMEM, "host allocation");
  s = build_plan(sys, o, pl);
  if (s != SAG_OK) {
    delete pl;
    return s;
  }
  *out = pl;
  return SAG_OK;
}

sag_status sag_plan_layout(sag_plan_t pl, int64_t* offsets) {
  if (!pl || !offsets) return fail(SAG_EINVAL, "NULL argument");
  offsets[0] = 0;
  offsets[1] = pl->N;
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
  const size_t nb = (size_t)pl->N * sizeof(double);
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
  sag_status s = eval(pl, nd, a, st);
  if (s != SAG_OK) return s;
  if (ph && (e = cudaMemcpyAsync(p, pl->stage_b, nb, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "copy p");
  if (qh && (e = cudaMemcpyAsync(q, pl->stage_c, nb, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "copy q");
  if (oh && (e = cudaMemcpyAsync(outflow, pl->dev_outflow, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "copy outflow");
  if (ph || qh || oh) {
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "sync");
  }
  return SAG_OK;
}

sag_status sag_rhs(sag_plan_t pl, const double* n, double* dndt, void* stream) {
  if (!pl || !n || !dndt) return fail(SAG_EINVAL, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nb = (size_t)pl->N * sizeof(double);
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
  sag_status s = eval(pl, nd, a, st);
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
  const size_t nb = (size_t)pl->N * sizeof(double);
  const bool h = !is_device_ptr(n);
  double* nd = n;
  cudaError_t e;
  if (h) {
    if ((e = cudaMemcpyAsync(pl->stage_a, n, nb, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_fail(e, "copy n");
    nd = pl->stage_a;
  }
  sag_status s = enqueue_step(pl, nd, dt, nullptr, st, true);
  if (s != SAG_OK) return s;
  if (h) {
    if ((e = cudaMemcpyAsync(n, pl->stage_a, nb, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "copy n back");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "sync");
  }
  return SAG_OK;
}

sag_status sag_integrate(sag_plan_t pl, double* n, double dt, int64_t steps, double* diag,
                         void* stream) {
  if (!pl || !n) return fail(SAG_EINVAL, "NULL argument");
  if (steps < 0) return fail(SAG_EINVAL, "steps must be >= 0");
  if (!std::isfinite(dt)) return fail(SAG_EINVAL, "dt is not finite");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nb = (size_t)pl->N * sizeof(double);
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
  const size_t dlen = (size_t)(steps + 1) * 3;
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

sag_status sag_sync_status(sag_plan_t pl, void* stream) {
  if (!pl) return fail(SAG_EINVAL, "NULL plan");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  unsigned int status = 0;
  if ((e = cudaMemcpy(&status, &pl->P.sc->status, sizeof(unsigned), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "read status");
  if (status) {
    unsigned int zero = 0;
    cudaMemcpy(&pl->P.sc->status, &zero, sizeof(unsigned), cudaMemcpyHostToDevice);
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

// Operation counts of the double-word arithmetic (FP32 instructions), as
// written in dw.cuh: dw_add 11, dw_mul 7, one component of a complex product
// (dot2) 19, so a complex add 22, a complex product 38, a real double-word
// constant times a complex 14, a power-of-two scale 4. FP64 arithmetic: a
// complex add 2, a complex product 4 (2 multiplies, 2 FMAs), a real times a
// complex 2.
struct OpCost {
  double cadd, cmul, kmul, scale;
};
static constexpr OpCost kCostDW{22, 38, 14, 4};
static constexpr OpCost kCostF64{2, 4, 2, 2};

static double dft_ops(int R, const OpCost& c) {
  switch (R) {
    case 2: return 2 * c.cadd;
    case 3: return 6 * c.cadd + c.kmul + c.scale;
    case 4: return 8 * c.cadd;
    case 5: return 16 * c.cadd + 8 * c.kmul;
    default: return 26 * c.cadd + 2 * c.kmul;  // radix 8: 8 + 2 + 16 adds, 2 constant products
  }
}

// One length-P transform with the given radix schedule.
static double fft_ops(int P, const radix_plan& rp, const OpCost& c) {
  double ops = 0.0;
  int Ns = 1;
  for (int s = 0; s < rp.n; ++s) {
    const int R = rp.r[s];
    ops += (double)(P / R) * (dft_ops(R, c) + (Ns > 1 ? (R - 1) * c.cmul : 0.0));
    Ns *= R;
  }
  return ops;
}

const char* sag_kernel_name(int32_t id) {
  static const char* names[KID_COUNT] = {"k_nmax", "k_nsplit", "k_dot", "k_fwd_col",
                                         "k_rows", "k_inv_col", "k_epilogue", "k_moments"};
  return (id >= 0 && id < KID_COUNT) ? names[id] : nullptr;
}

sag_status sag_kernel_work(sag_plan_t pl, int32_t id, double* ops, int32_t* ops_fp64, double* bytes) {
  if (!pl || !ops || !ops_fp64 || !bytes) return fail(SAG_EINVAL, "NULL argument");
  if (id < 0 || id >= KID_COUNT) return fail(SAG_EINVAL, "kernel id out of range");
  const RhsParams& P = pl->P;
  const bool dwp = P.dwpath != 0;
  const OpCost& c = dwp ? kCostDW : kCostF64;
  const double N = P.N, V = P.Vtot;
  const double load_mul = dwp ? 7.0 : 1.0;  // a = U n: dw_mul or one FP64 multiply
  double o = 0.0, b = 0.0;
  int fp64 = dwp ? 0 : 1;
  switch (id) {
    case KID_NMAX:
      o = 2 * N;
      b = 8 * N;
      fp64 = 1;
      break;
    case KID_NSPLIT:
      o = 4 * N;
      b = 16 * N;
      fp64 = 1;
      break;
    case KID_DOT:  // u n, sum, k (u n) + t
      o = 3 * V * N;
      b = 8 * V * N + 8 * N;
      fp64 = 1;
      break;
    case KID_FWD_COL:
      for (int i = 0; i < P.nord; ++i) {
        const OrderDesc& od = P.ord[i];
        const double Vd = (double)od.d * od.R;
        o += Vd * (od.M2 * fft_ops(od.M1, od.rp1, c) + (double)od.M * c.cmul +
                   2.0 * std::min<double>(od.M, N) * load_mul);
      }
      b = (dwp ? 8.0 : 8.0) * V * N + (dwp ? 8.0 : 8.0) * N;
      break;
    case KID_ROWS:
      for (int i = 0; i < P.nord; ++i) {
        const OrderDesc& od = P.ord[i];
        const double Vd = (double)od.d * od.R, M = od.M;
        const double unpack = 4 * c.cadd + c.cmul;
        const double repack = 4 * c.cadd + c.cmul;
        o += Vd * od.M1 * fft_ops(od.M2, od.rp2, c)            // forward rows of every vector
             + Vd * M * unpack                                   // real split
             + (Vd - od.R) * M * c.cmul                          // product over the modes
             + (double)od.R * M * (c.cadd + (dwp ? c.scale : 0)) // rank sum
             + M * repack + od.M1 * fft_ops(od.M2, od.rp2, c)    // inverse rows
             + M * c.cmul;                                       // four-step twiddle
      }
      b = 0.0;  // reads and writes only the FFT workspace
      break;
    case KID_INV_COL:
      for (int i = 0; i < P.nord; ++i) {
        const OrderDesc& od = P.ord[i];
        o += od.M2 * fft_ops(od.M1, od.rp1, c);
      }
      b = 8.0 * P.nord * N;  // P^(d) written
      break;
    case KID_EPILOGUE:  // w = sum_v coef_v U_v(k); rhs = p + n w; stage update
      o = V * N + (P.nord + 6) * N;
      b = 8 * V * N + 8 * P.nord * N + 3 * 8 * N;
      fp64 = 1;
      break;
    case KID_MOMENTS:
      o = 3 * N;
      b = 8 * N;
      fp64 = 1;
      break;
  }
  *ops = o;
  *ops_fp64 = fp64;
  *bytes = b;
  return SAG_OK;
}

sag_status sag_plan_describe(sag_plan_t pl, char* buf, size_t len) {
  if (!pl || !buf || len == 0) return fail(SAG_EINVAL, "NULL argument");
  const RhsParams& P = pl->P;
  std::string js = "{\"N\": " + std::to_string(P.N) + ", \"D\": " + std::to_string(P.D) +
                   ", \"precision\": \"" + (P.dwpath ? "fp32_split" : "fp64") + "\", \"orders\": [";
  for (int i = 0; i < P.nord; ++i) {
    const OrderDesc& od = P.ord[i];
    auto rps = [](const radix_plan& rp) {
      std::string r = "[";
      for (int s = 0; s < rp.n; ++s) r += (s ? ", " : "") + std::to_string(rp.r[s]);
      return r + "]";
    };
    js += std::string(i ? ", " : "") + "{\"d\": " + std::to_string(od.d) + ", \"R\": " +
          std::to_string(od.R) + ", \"L\": " + std::to_string(od.L) + ", \"M1\": " +
          std::to_string(od.M1) + ", \"M2\": " + std::to_string(od.M2) + ", \"radix_M1\": " +
          rps(od.rp1) + ", \"radix_M2\": " + rps(od.rp2) + ", \"W\": " + std::to_string(od.W) +
          ", \"G\": " + std::to_string(od.G) + "}";
  }
  js += "], \"blocks\": {\"fwd_col\": " + std::to_string(pl->L.col_blocks) + ", \"rows\": " +
        std::to_string(pl->L.row_blocks) + ", \"inv_col\": " + std::to_string(pl->L.inv_blocks) +
        ", \"epilogue\": " + std::to_string(pl->L.epi_blocks) + "}, \"device_bytes\": " +
        std::to_string(pl->bytes) + "}";
  std::snprintf(buf, len, "%s", js.c_str());
  return SAG_OK;
}

void sag_plan_destroy(sag_plan_t pl) {
  if (!pl) return;
  cudaDeviceSynchronize();
  delete pl;
}

}  // extern "C"
