// Loss term without any device allocation.
//
// sag_loss_noalloc evaluates q = sum_d Q^(d)[n] for a CP system straight from
// caller-owned device buffers, for callers that cannot call cudaMalloc (code
// running under an allocator it does not own, inside a memory pool with a fixed
// budget, or in a process whose device memory was reserved up front). The
// per-chunk partial inner products that the plan-based path keeps in its
// workspace live here in one file-scope device array instead, so the call
// allocates nothing: no cudaMalloc, no cudaFree, no allocating library routine.
#include <cuda_runtime.h>

#include <mutex>

#include "launch.h"
#include "sag.h"

namespace sag {
sag_status set_last_error(sag_status s, const char* msg);
}

namespace {

constexpr int kLossChunk = 8192;          // sizes per partial sum
constexpr int kLossMaxPartials = 32768;   // V * ceil(N / 8192) partials at most (256 KB)
constexpr int kLossMaxVectors = 2048;     // V = sum_d d R_d at most (shared-memory weights)
constexpr int kMaxDevices = 64;

// Every device that loads the library holds this array until the process exits:
// kLossMaxPartials partial inner products, then kLossMaxVectors loss weights
// coef_v (288 KB in all). Each call overwrites every entry it later reads, so
// nothing in it has to start at zero; concurrent calls (overlapping on any
// stream) race on it.
static __device__ __align__(256) double g_loss_partials[kLossMaxPartials + kLossMaxVectors];

std::mutex g_mu;
double* g_partials_addr[kMaxDevices] = {};

struct LossDesc {
  int N, nord, V, nchunk, sym;
  int d[sag::kMaxD], R[sag::kMaxD], vbase[sag::kMaxD];
};

// Partial sums of s_v = <U_v, n> over one chunk of sizes (FP64, warp shuffles).
__global__ void __launch_bounds__(256) k_loss_partials(LossDesc L, const double* __restrict__ U,
                                                       const double* __restrict__ n,
                                                       double* __restrict__ part) {
  __shared__ double red[32];
  const int v = blockIdx.y, c = blockIdx.x;
  const int k0 = c * kLossChunk, k1 = min(L.N, k0 + kLossChunk);
  const double* u = U + (int64_t)v * L.N;
  double acc = 0.0;
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) acc += u[k] * n[k];
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) part[v * L.nchunk + c] = acc;
  }
}

// One block: s_v = sum of vector v's chunk partials, then the loss weights
// coef_v = -1/(d-1)! (1/d) prod_{m' != m} s_{d,m',r} (symmetrised) or
// -1/(d-1)! [m = d-1] prod_{m' < d-1} s_{d,m',r} (last mode), written after
// the partials.
__global__ void __launch_bounds__(256) k_loss_coef(LossDesc L, const double* __restrict__ part,
                                                   double* __restrict__ coef) {
  extern __shared__ double s[];
  for (int v = threadIdx.x; v < L.V; v += blockDim.x) {
    double a = 0.0;
    for (int c = 0; c < L.nchunk; ++c) a += part[v * L.nchunk + c];
    s[v] = a;
  }
  __syncthreads();
  for (int v = threadIdx.x; v < L.V; v += blockDim.x) {
    int oi = 0;
    while (oi + 1 < L.nord && v >= L.vbase[oi + 1]) ++oi;
    const int d = L.d[oi], R = L.R[oi], loc = v - L.vbase[oi], m = loc / R, r = loc - m * R;
    double prod = 1.0;
    for (int mm = 0; mm < d; ++mm)
      if (mm != m) prod *= s[L.vbase[oi] + mm * R + r];
    double f = 1.0;
    for (int i = 2; i <= d - 1; ++i) f *= i;
    const double c = L.sym ? prod / d : (m == d - 1 ? prod : 0.0);
    coef[v] = -c / f;
  }
}

// q_k = n_k sum_v coef_v U_v(k).
__global__ void __launch_bounds__(256) k_loss_assemble(LossDesc L, const double* __restrict__ U,
                                                       const double* __restrict__ n,
                                                       const double* __restrict__ coef_g,
                                                       double* __restrict__ q) {
  extern __shared__ double coef[];
  for (int v = threadIdx.x; v < L.V; v += blockDim.x) coef[v] = coef_g[v];
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < L.N) {
    double w = 0.0;
    for (int v = 0; v < L.V; ++v) w = fma(coef[v], U[(int64_t)v * L.N + k], w);
    q[k] = n[k] * w;
  }
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" sag_status sag_loss_noalloc(const sag_system* sys, int32_t symmetrize_q, const double* n,
                                       double* q, void* stream) {
  using sag::set_last_error;
  if (!sys || !n || !q || !sys->rank || !sys->factors) return set_last_error(SAG_EINVAL, "NULL argument");
  if (sys->fmt != SAG_CP) return set_last_error(SAG_EUNSUPPORTED, "sag_loss_noalloc takes CP kernels only");
  if (sys->N < 1 || sys->D < 2 || sys->D > sag::kMaxD) return set_last_error(SAG_EINVAL, "N >= 1 and 2 <= D <= 8 required");
  if (symmetrize_q != 0 && symmetrize_q != 1) return set_last_error(SAG_EINVAL, "symmetrize_q must be 0 or 1");
  LossDesc L{};
  L.N = sys->N;
  L.sym = symmetrize_q;
  // As in sag_plan, a CP rank of 0 leaves an order out, and at least one order
  // needs a rank of 1 or more.
  int64_t V = 0;
  for (int d = 2; d <= sys->D; ++d) {
    const int R = sys->rank[d - 2];
    if (R < 0) return set_last_error(SAG_EINVAL, "CP ranks must be >= 0");
    if (R == 0) continue;
    L.d[L.nord] = d;
    L.R[L.nord] = R;
    L.vbase[L.nord] = (int)V;
    ++L.nord;
    V += (int64_t)d * R;
    if (V > kLossMaxVectors) break;
  }
  if (L.nord == 0) return set_last_error(SAG_EINVAL, "every system needs one order of CP rank >= 1");
  L.nchunk = (L.N + kLossChunk - 1) / kLossChunk;
  if (V > kLossMaxVectors || V * L.nchunk > kLossMaxPartials)
    return set_last_error(SAG_EINVAL,
                          "system too large for sag_loss_noalloc: needs sum_d d R_d <= 2048 and "
                          "(sum_d d R_d) * ceil(N / 8192) <= 32768");
  L.V = (int)V;
  if (!sys->factors_on_device || !on_device(sys->factors) || !on_device(n) || !on_device(q))
    return set_last_error(SAG_EINVAL, "sag_loss_noalloc needs device pointers for factors, n and q");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_last_error(SAG_ECUDA, "cudaGetDevice failed or device index out of range");
  double* part = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_partials_addr[dev]) {
      // Once per device, with that device current: the device address of the
      // static array (its name in host code is only a host-side stand-in).
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_loss_partials);
      if (e != cudaSuccess) return set_last_error(SAG_ECUDA, "cudaGetSymbolAddress failed");
      g_partials_addr[dev] = static_cast<double*>(p);
    }
    part = g_partials_addr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* coef = part + kLossMaxPartials;
  k_loss_partials<<<dim3(L.nchunk, L.V), 256, 0, st>>>(L, sys->factors, n, part);
  k_loss_coef<<<1, 256, L.V * sizeof(double), st>>>(L, part, coef);
  k_loss_assemble<<<(L.N + 255) / 256, 256, L.V * sizeof(double), st>>>(L, sys->factors, n, coef, q);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_last_error(SAG_ECUDA, cudaGetErrorString(e));
  return SAG_OK;
}
