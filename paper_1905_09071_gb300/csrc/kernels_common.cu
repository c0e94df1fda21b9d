// Kernels of the right-hand side that are not FFTs: the double-word scaling of
// n, the loss-term inner products, and the epilogue that assembles
// dn/dt = P + Q and applies the Runge-Kutta stage update.
#include "launch.h"

namespace sag {

// ---- block reductions (fixed order, hence deterministic) -------------------
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /* 32 * NV */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    for (int o = 16; o; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[warp * NV + i] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      v[i] = lane < nw ? sh[lane * NV + i] : 0.0;
      for (int o = 16; o; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
  }
  __syncthreads();
}

// ---- n for the double-word path: n * 2^-e_n with max |n| 2^-e_n in [0.5, 1) --
__global__ void k_nmax(const double* __restrict__ n, int N, DevScalars* sc) {
  double m = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x)
    m = fmax(m, fabs(n[k]));
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0)
    atomicMax(&sc->nmax_bits, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_nsplit(const double* __restrict__ n, int N, DevScalars* sc, float2* ndw) {
  const double mx = __longlong_as_double((long long)sc->nmax_bits);
  const int e = (mx > 0.0 && isfinite(mx)) ? ilogb(mx) + 1 : 0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    const dw v = dw_from_double(scalbn(n[k], -e));
    ndw[k] = make_float2(v.hi, v.lo);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->e_n = e;
}

// ---- loss-term inner products (Sec. 1: the (d-1)-fold sums of q^(d) split
// into products of s_{d,m,r} = <U^(m)_r, n> for a CP kernel), FP64, plus the
// first moments t = <k U^(m)_r, n> used for the outflow diagnostic. --------
__global__ void __launch_bounds__(256) k_dot(const __grid_constant__ RhsParams P,
                                             const double* __restrict__ n) {
  __shared__ double sh[64];
  const int v = blockIdx.y, c = blockIdx.x;
  const int k0 = c * P.dotchunk, k1 = min(P.N, k0 + P.dotchunk);
  const double* u = P.U64 + (int64_t)v * P.N;
  double acc[2] = {0.0, 0.0};
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const double un = u[k] * n[k];
    acc[0] += un;
    acc[1] = fma((double)(k + 1), un, acc[1]);
  }
  block_sum<2>(acc, sh);
  if (threadIdx.x == 0) {
    P.dot_s[v * P.ndotchunk + c] = acc[0];
    P.dot_t[v * P.ndotchunk + c] = acc[1];
  }
}

// Order index of a global vector.
__device__ __forceinline__ int order_of_vector(const RhsParams& P, int v) {
  int oi = 0;
  while (oi + 1 < P.nord && v >= P.ord[oi + 1].vbase) ++oi;
  return oi;
}

__device__ __forceinline__ double inv_factorial(int d) {
  double f = 1.0;
  for (int i = 2; i <= d; ++i) f *= i;
  return 1.0 / f;
}

// ---- epilogue --------------------------------------------------------------
// Every block first reduces the inner products s_v and turns them into the
// loss weights: q_k = n_k sum_v coef_v U_v(k) with, for v = (d, m, r),
//   coef_v = -1/(d-1)! * (1/d) prod_{m' != m} s_{d,m',r}   (symmetrised kernel)
//   coef_v = -1/(d-1)! * [m = d-1] prod_{m' < d-1} s_{d,m',r}   (literal, last mode)
// The last block to finish reduces the block partials and evaluates the
// outflow sum_d 1/d! sum_{i in [1,N]^d} |i| C_i prod n  -  sum_{k<=N} k P_k,
// whose first part is sum_r sum_m t_{d,m,r} prod_{m' != m} s_{d,m',r} / d!.
__global__ void __launch_bounds__(256) k_epilogue(const __grid_constant__ RhsParams P, EpiArgs A) {
  extern __shared__ double esh[];  // [Vtot] s, [Vtot] coef
  __shared__ double red[32 * 4];
  __shared__ int is_last;
  double* s = esh;
  double* coef = esh + P.Vtot;
  const int N = P.N, V = P.Vtot, nc = P.ndotchunk;
  for (int v = threadIdx.x; v < V; v += blockDim.x) {
    double a = 0.0;
    for (int c = 0; c < nc; ++c) a += P.dot_s[v * nc + c];
    s[v] = a;
  }
  __syncthreads();
  for (int v = threadIdx.x; v < V; v += blockDim.x) {
    const int oi = order_of_vector(P, v);
    const OrderDesc& od = P.ord[oi];
    const int d = od.d, R = od.R, loc = v - od.vbase, m = loc / R, r = loc - m * R;
    double prod = 1.0;
    for (int mm = 0; mm < d; ++mm)
      if (mm != m) prod *= s[od.vbase + mm * R + r];
    double c;
    if (P.sym) c = prod / d;
    else c = (m == d - 1) ? prod : 0.0;
    coef[v] = -inv_factorial(d - 1) * c;
  }
  __syncthreads();

  double part[3] = {0.0, 0.0, 0.0};  // sum k p_k, M0 and M1 of the new state
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) {
    double p = 0.0;
    for (int oi = 0; oi < P.nord; ++oi) p += P.pd[(int64_t)oi * N + k];
    double w = 0.0;
    for (int v = 0; v < V; ++v) w = fma(coef[v], P.U64[(int64_t)v * N + k], w);
    const double nk = A.nin[k];
    const double q = nk * w;
    const double rhs = p + q;
    if (!isfinite(rhs)) atomicOr(&P.sc->status, kStatusNonFinite);
    const double size = (double)(k + 1);
    part[0] = size * p;
    double nn = 0.0;
    switch (A.mode) {
      case EPI_RHS:
        if (A.out0) A.out0[k] = rhs;
        if (A.pout) A.pout[k] = p;
        if (A.qout) A.qout[k] = q;
        break;
      case EPI_HEUN1:
        A.k1buf[k] = rhs;
        A.out0[k] = nk + A.dt * rhs;
        break;
      case EPI_MID1:
        A.out0[k] = nk + 0.5 * A.dt * rhs;
        break;
      case EPI_HEUN2:
        nn = A.nbase[k] + 0.5 * A.dt * (A.k1buf[k] + rhs);
        A.nbase[k] = nn;
        break;
      case EPI_MID2:
        nn = A.nbase[k] + A.dt * rhs;
        A.nbase[k] = nn;
        break;
    }
    part[1] = nn;
    part[2] = size * nn;
  }
  block_sum<3>(part, red);
  if (threadIdx.x == 0) {
    A.part[blockIdx.x * 4 + 0] = part[0];
    A.part[blockIdx.x * 4 + 1] = part[1];
    A.part[blockIdx.x * 4 + 2] = part[2];
    __threadfence();
    const unsigned ticket = atomicAdd(&P.sc->counter, 1u);
    is_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();

  // Last block: fixed-order reduction of the block partials and of the
  // outflow's complete-sum term.
  double tot[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    tot[0] += __ldcg(&A.part[b * 4 + 0]);
    tot[1] += __ldcg(&A.part[b * 4 + 1]);
    tot[2] += __ldcg(&A.part[b * 4 + 2]);
  }
  for (int v = threadIdx.x; v < V; v += blockDim.x) {
    const int oi = order_of_vector(P, v);
    const OrderDesc& od = P.ord[oi];
    const int d = od.d, R = od.R, loc = v - od.vbase, m = loc / R, r = loc - m * R;
    double t = 0.0;
    for (int c = 0; c < nc; ++c) t += P.dot_t[v * nc + c];
    double prod = 1.0;
    for (int mm = 0; mm < d; ++mm)
      if (mm != m) prod *= s[od.vbase + mm * R + r];
    tot[3] += t * prod * inv_factorial(d);
  }
  block_sum<4>(tot, red);
  if (threadIdx.x == 0) {
    DevScalars* sc = P.sc;
    const double outflow = tot[3] - tot[0];
    sc->outflow = outflow;
    switch (A.mode) {
      case EPI_RHS:
        if (A.outflow_out) *A.outflow_out = outflow;
        break;
      case EPI_HEUN1:
        sc->o_stage1 = outflow;
        break;
      case EPI_MID1:
        break;
      case EPI_HEUN2:
      case EPI_MID2: {
        sc->cum += (A.mode == EPI_HEUN2) ? 0.5 * A.dt * (sc->o_stage1 + outflow) : A.dt * outflow;
        const int row = ++sc->step;
        if (A.diag) {
          A.diag[row * 3 + 0] = tot[1];
          A.diag[row * 3 + 1] = tot[2];
          A.diag[row * 3 + 2] = sc->cum;
        }
        break;
      }
    }
    sc->counter = 0u;
    sc->nmax_bits = 0ull;
  }
}

// Row 0 of the diagnostics (M0, M1 of n, zero outflow) and the integrator's
// counters. One block.
__global__ void __launch_bounds__(256) k_moments(const double* __restrict__ n, int N, DevScalars* sc,
                                                 double* diag) {
  __shared__ double red[64];
  double acc[2] = {0.0, 0.0};
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    acc[0] += n[k];
    acc[1] = fma((double)(k + 1), n[k], acc[1]);
  }
  block_sum<2>(acc, red);
  if (threadIdx.x == 0) {
    sc->step = 0;
    sc->cum = 0.0;
    if (diag) {
      diag[0] = acc[0];
      diag[1] = acc[1];
      diag[2] = 0.0;
    }
  }
}

// ---- launch of one evaluation ---------------------------------------------
cudaError_t enqueue_eval(const RhsParams& P, const LaunchCfg& L, const double* nin,
                         const EpiArgs& A, cudaStream_t st, LaunchHook* hook) {
  if (P.dwpath) {
    if (hook) hook->mark(KID_NMAX, st);
    k_nmax<<<L.prep_blocks, 256, 0, st>>>(nin, P.N, P.sc);
    if (hook) hook->mark(KID_NSPLIT, st);
    k_nsplit<<<L.prep_blocks, 256, 0, st>>>(nin, P.N, P.sc, P.ndw);
  }
  if (hook) hook->mark(KID_DOT, st);
  k_dot<<<dim3(P.ndotchunk, P.Vtot), 256, 0, st>>>(P, nin);
  cudaError_t e = P.dwpath ? enqueue_fft_dw(P, L, nin, st, hook) : enqueue_fft_f64(P, L, nin, st, hook);
  if (e != cudaSuccess) return e;
  if (hook) hook->mark(KID_EPILOGUE, st);
  k_epilogue<<<L.epi_blocks, 256, L.epi_smem, st>>>(P, A);
  if (hook) hook->mark(-1, st);
  return cudaGetLastError();
}

cudaError_t enqueue_moments(const RhsParams& P, const double* n, double* diag, cudaStream_t st) {
  k_moments<<<1, 256, 0, st>>>(n, P.N, P.sc, diag);
  return cudaGetLastError();
}

cudaError_t setup_common_kernels(const LaunchCfg& L) {
  return cudaFuncSetAttribute(k_epilogue, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.epi_smem);
}

}  // namespace sag
