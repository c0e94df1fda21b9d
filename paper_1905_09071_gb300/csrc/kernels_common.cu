// Kernels of the right-hand side that are not FFTs: the double-word scaling of
// n, the loss-term inner products and weights, and the epilogue that
// assembles dn/dt = P + Q and applies the Runge-Kutta stage update. Every
// kernel covers all systems of the plan in one launch.
#include "dw_pow.cuh"
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

__device__ __forceinline__ double inv_factorial(int d) {
  double f = 1.0;
  for (int i = 2; i <= d; ++i) f *= i;
  return 1.0 / f;
}

// ---- n for the double-word path: per system, n 2^-e_n with max |n| 2^-e_n in
// [0.5, 1) (an exact power-of-two scale). Grid: (blocks per system, B).
__global__ void k_nmax(const __grid_constant__ RhsParams P, const double* __restrict__ n) {
  const SysDesc s = P.sys[blockIdx.y];
  const double* x = n + s.noff;
  double m = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < s.N; k += gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[k]));
  // one atomic per block (warps, then the block's first warp)
  __shared__ double wm[32];
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? wm[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0 && m > 0.0)
      atomicMax(&P.sc[blockIdx.y].nmax_bits, (unsigned long long)__double_as_longlong(m));
  }
}

__global__ void k_nsplit(const __grid_constant__ RhsParams P, const double* __restrict__ n) {
  const SysDesc s = P.sys[blockIdx.y];
  SysScalars* sc = &P.sc[blockIdx.y];
  const double mx = __longlong_as_double((long long)sc->nmax_bits);
  const int e = (mx > 0.0 && isfinite(mx)) ? ilogb(mx) + 1 : 0;
  const double* x = n + s.noff;
  float2* out = P.ndw + s.ndwoff + 1;  // element index = size
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < s.N; k += gridDim.x * blockDim.x) {
    const dw v = dw_from_double(scalbn(x[k], -e));
    out[k] = make_float2(v.hi, v.lo);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->e_n = e;
}

// ---- loss-term inner products (Sec. 1: for a low-rank kernel the (d-1)-fold
// sums of q^(d) split into products of s_v = <U_v, n>), FP64, plus the first
// moments t_v = <k U_v, n> used by the outflow diagnostic. Per thread the sizes
// k_i = base + 256 i are visited in decreasing i with x_i = U(k_i) n(k_i):
// acc1 = sum x_i and acc2 = sum (i + 1) x_i (a running sum of running sums),
// so t = base acc1 + 256 (acc2 - acc1) costs one FMA and one add per size.
// Grid: (vectors, most chunks of any vector).
// The first moments t are needed only for the outflow diagnostic (flux = 1);
// without them the kernel does half the FP64 work.
__global__ void __launch_bounds__(256) k_dot(const __grid_constant__ RhsParams P,
                                             const double* __restrict__ n, int flux) {
  __shared__ double sh[64];
  const int v = blockIdx.x, c = blockIdx.y;
  if (P.vrep[v] != v) return;  // a repeated vector: the first of its set has the sums
  const SysDesc s = P.sys[P.vsys[v]];
  if (c >= s.ndotchunk) return;
  const int k0 = c * P.dotchunk, k1 = min(s.N, k0 + P.dotchunk);
  const double* u = P.U64 + P.voff[v];
  const double* x = n + s.noff;
  const int first = k0 + threadIdx.x;
  const int cnt = first < k1 ? (k1 - first + 255) / 256 : 0;
  double acc1 = 0.0, acc2 = 0.0;
  if (flux) {
    for (int i = cnt - 1; i >= 0; --i) {
      const int k = first + i * 256;
      acc1 = fma(u[k], x[k], acc1);
      acc2 += acc1;
    }
  } else {
    for (int i = cnt - 1; i >= 0; --i) acc1 = fma(u[first + i * 256], x[first + i * 256], acc1);
  }
  if (flux) {
    double acc[2] = {acc1, (double)(first + 1) * acc1 + 256.0 * (acc2 - acc1)};
    block_sum<2>(acc, sh);
    if (threadIdx.x == 0) {
      P.dot_s[(int64_t)v * P.maxdotchunk + c] = acc[0];
      P.dot_t[(int64_t)v * P.maxdotchunk + c] = acc[1];
    }
  } else {  // one reduction instead of two: the FP64 adds of the tree count
    double acc[1] = {acc1};
    block_sum<1>(acc, sh);
    if (threadIdx.x == 0) P.dot_s[(int64_t)v * P.maxdotchunk + c] = acc[0];
  }
}

// ---- loss weights and the complete first-moment flux, one block per system --
// q_k = n_k sum_v coef_v U_v(k). For a CP vector v = (d, m, r):
//   coef_v = -1/(d-1)! (1/d) prod_{m' != m} s_{d,m',r}   (symmetrised kernel)
//   coef_v = -1/(d-1)! [m = d-1] prod_{m' < d-1} s_{d,m',r}   (last mode)
// For a TT vector v = h^(l)_{a,b} of order d, with M_l[a][b] = s of h^(l)_{a,b}:
//   coef_v = -1/(d-1)! w_l (e_0 M_1 ... M_{l-1})[a] (M_{l+1} ... M_d e_0)[b],
//   w_l = 1/d (symmetrised) or [l = d] (last mode).
// gflux = sum_d 1/d! sum_{i in [1,N]^d} |i| C_i prod n: the same products with
// one s replaced by the first moment t (only with flux = 1; else t = 0 and
// gflux = 0, and the outflow derived from it is not meaningful).
__global__ void __launch_bounds__(256) k_coef(const __grid_constant__ RhsParams P, int flux) {
  extern __shared__ double csh[];  // [vectors of the system] s, then t
  __shared__ double red[32];
  const int b = blockIdx.x;
  const SysDesc sy = P.sys[b];
  const int nv = sy.vend - sy.vbeg, nc = sy.ndotchunk;
  double* s = csh;
  double* t = csh + nv;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const int64_t base = (int64_t)P.vrep[sy.vbeg + i] * P.maxdotchunk;  // repeats: the first's sums
    double a = 0.0, c2 = 0.0;
    for (int c = 0; c < nc; ++c) {
      a += P.dot_s[base + c];
      if (flux) c2 += P.dot_t[base + c];
    }
    s[i] = a;
    t[i] = c2;
  }
  __syncthreads();
  double g[1] = {0.0};
  if (sy.fmt == 0) {
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
      const int v = sy.vbeg + i;
      int it = sy.ibeg;
      while (it + 1 < sy.iend && v >= P.ord[it + 1].vbase) ++it;
      const OrderDesc od = P.ord[it];
      const int d = od.d, R = od.R, loc = v - od.vbase, m = loc / R, r = loc - m * R;
      const int lb = od.vbase - sy.vbeg;
      double prod = 1.0;
      for (int mm = 0; mm < d; ++mm)
        if (mm != m) prod *= s[lb + mm * R + r];
      const double c = P.sym ? prod / d : (m == d - 1 ? prod : 0.0);
      P.coef[v] = -inv_factorial(d - 1) * c;
      g[0] += t[i] * prod * inv_factorial(d);
    }
  } else if (threadIdx.x < sy.iend - sy.ibeg) {
    // One thread per order: left and right products of the inner-product matrices.
    const OrderDesc od = P.ord[sy.ibeg + threadIdx.x];
    const int d = od.d;
    const int* vid = P.vid + od.vid_off;
    double left[kMaxD + 1][kMaxTTRank], right[kMaxD + 1][kMaxTTRank];
    int offs[kMaxD + 1];
    // left[l] = e_0 M_1 ... M_l (length R_l); right[l] = M_{l+1} ... M_d e_0 (length R_l)
    left[0][0] = 1.0;
    int off = 0;
    for (int l = 1; l <= d; ++l) {
      offs[l] = off;
      const int ra = od.ttr[l - 1], rb = od.ttr[l];
      for (int bb = 0; bb < rb; ++bb) {
        double acc = 0.0;
        for (int a = 0; a < ra; ++a) {
          const int w = vid[off + a * rb + bb];
          if (w >= 0) acc += left[l - 1][a] * s[w - sy.vbeg];
        }
        left[l][bb] = acc;
      }
      off += ra * rb;
    }
    right[d][0] = 1.0;
    for (int l = d; l >= 1; --l) {
      const int ra = od.ttr[l - 1], rb = od.ttr[l];
      for (int a = 0; a < ra; ++a) {
        double acc = 0.0;
        for (int bb = 0; bb < rb; ++bb) {
          const int w = vid[offs[l] + a * rb + bb];
          if (w >= 0) acc += s[w - sy.vbeg] * right[l][bb];
        }
        right[l - 1][a] = acc;
      }
    }
    // Core entries that share a vector (bitwise-identical entries of the
    // order's cores) add their weights; this thread owns the order's vectors.
    for (int v = od.vbase; v < od.vbase + od.nvec; ++v) P.coef[v] = 0.0;
    for (int l = 1; l <= d; ++l) {
      const int ra = od.ttr[l - 1], rb = od.ttr[l];
      const double wl = P.sym ? 1.0 / d : (l == d ? 1.0 : 0.0);
      for (int a = 0; a < ra; ++a)
        for (int bb = 0; bb < rb; ++bb) {
          const int w = vid[offs[l] + a * rb + bb];
          if (w < 0) continue;
          const double lr = left[l - 1][a] * right[l][bb];
          P.coef[w] += -inv_factorial(d - 1) * wl * lr;
          g[0] += t[w - sy.vbeg] * lr * inv_factorial(d);
        }
    }
  }
  block_sum<1>(g, red);
  if (threadIdx.x == 0) P.sc[b].gflux = g[0];
}

// ---- epilogue --------------------------------------------------------------
// rhs_k = sum_d P^(d)_k + n_k sum_v coef_v U_v(k), then the Runge-Kutta stage.
// The last block of each system to finish reduces that system's block
// partials in a fixed order and evaluates its outflow gflux - sum_{k<=N} k P_k.
// q_k = n_k sum_v coef_v U_v(k): one pass over the FP64 factors. It needs
// only the loss weights, so it runs on the side branch beside the FFT kernels.
__global__ void __launch_bounds__(256) k_qterm(const __grid_constant__ RhsParams P,
                                               const double* __restrict__ nin) {
  extern __shared__ double esh[];  // [vectors of the system] coef, then folded weights
  const int b = find_segment(P.epipre, P.B, blockIdx.x);
  const SysDesc sy = P.sys[b];
  const int blk = blockIdx.x - P.epipre[b];
  const int nv = sy.vend - sy.vbeg, N = sy.N, nd = sy.dend - sy.dbeg;
  double* coef = esh;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) coef[i] = P.coef[sy.vbeg + i];
  __syncthreads();
  const int k = blk * blockDim.x + threadIdx.x;
  if (nd < nv) {
    // Repeated vectors: the weights of each set added (in vector order) onto
    // its first vector, then one pass over the distinct vectors.
    double* wsum = esh + nv;
    for (int j = threadIdx.x; j < nd; j += blockDim.x) {
      const int u = P.vdist[sy.dbeg + j];
      double a = 0.0;
      for (int i = 0; i < nv; ++i)
        if (P.vrep[sy.vbeg + i] == u) a += coef[i];
      wsum[j] = a;
    }
    __syncthreads();
    if (k >= N) return;
    const double* Ub = P.U64 + P.voff[sy.vbeg] + k;  // a system's vectors are back to back
    double w0 = 0.0, w1 = 0.0;
    int j = 0;
    for (; j + 1 < nd; j += 2) {
      w0 = fma(wsum[j], Ub[(int64_t)(P.vdist[sy.dbeg + j] - sy.vbeg) * N], w0);
      w1 = fma(wsum[j + 1], Ub[(int64_t)(P.vdist[sy.dbeg + j + 1] - sy.vbeg) * N], w1);
    }
    if (j < nd) w0 = fma(wsum[j], Ub[(int64_t)(P.vdist[sy.dbeg + j] - sy.vbeg) * N], w0);
    const int64_t g = sy.noff + k;
    P.qbuf[g] = nin[g] * (w0 + w1);
    return;
  }
  if (k >= N) return;
  // A system's vectors are stored back to back, N sizes each.
  const double* Ub = P.U64 + P.voff[sy.vbeg] + k;
  double w0 = 0.0, w1 = 0.0;
  int i = 0;
  for (; i + 1 < nv; i += 2) {
    w0 = fma(coef[i], Ub[(int64_t)i * N], w0);
    w1 = fma(coef[i + 1], Ub[(int64_t)(i + 1) * N], w1);
  }
  if (i < nv) w0 = fma(coef[i], Ub[(int64_t)i * N], w0);
  const int64_t g = sy.noff + k;
  P.qbuf[g] = nin[g] * (w0 + w1);
}

__global__ void __launch_bounds__(256) k_epilogue(const __grid_constant__ RhsParams P, EpiArgs A) {
  __shared__ double red[32 * 4];
  __shared__ int is_last;
  const int b = find_segment(P.epipre, P.B, blockIdx.x);
  const SysDesc sy = P.sys[b];
  const int blk = blockIdx.x - P.epipre[b];
  const int N = sy.N;

  double part[3] = {0.0, 0.0, 0.0};  // sum k p_k, M0 and M1 of the new state
  const int k = blk * blockDim.x + threadIdx.x;
  if (k < N) {
    const int64_t g = sy.noff + k;
    double p = 0.0;
    for (int it = sy.ibeg; it < sy.iend; ++it) p += P.pd[P.ord[it].pd_off + k];
    const double nk = A.nin[g];
    const double q = P.qbuf[g];
    const double rhs = p + q;
    if (!isfinite(rhs)) atomicOr(P.status, kStatusNonFinite);
    const double size = (double)(k + 1);
    part[0] = size * p;
    double nn = 0.0;
    switch (A.mode) {
      case EPI_RHS:
        if (A.out0) A.out0[g] = rhs;
        if (A.pout) A.pout[g] = p;
        if (A.qout) A.qout[g] = q;
        break;
      case EPI_HEUN1:
        A.k1buf[g] = rhs;
        nn = nk + A.dt * rhs;
        A.out0[g] = nn;
        break;
      case EPI_MID1:
        nn = nk + 0.5 * A.dt * rhs;
        A.out0[g] = nn;
        break;
      case EPI_HEUN2:
        nn = A.nbase[g] + 0.5 * A.dt * (A.k1buf[g] + rhs);
        A.nbase[g] = nn;
        break;
      case EPI_MID2:
        nn = A.nbase[g] + A.dt * rhs;
        A.nbase[g] = nn;
        break;
    }
    if (A.split_next) {
      // the stage state's double-word copy for the next evaluation, at this
      // evaluation's scale 2^-e_n (the next one skips k_nmax and k_nsplit)
      const dw v = dw_from_double(scalbn(nn, -P.sc[b].e_n));
      P.ndw[sy.ndwoff + 1 + k] = make_float2(v.hi, v.lo);
    }
    part[1] = nn;
    part[2] = size * nn;
  }
  SysScalars* sc = &P.sc[b];
  if (!A.flux) {
    // No diagnostics or outflow wanted: no moment sums. Clear the max of n for
    // the next evaluation's k_nmax (this evaluation's k_nsplit has run).
    if (blk == 0 && threadIdx.x == 0) sc->nmax_bits = 0ull;
    return;
  }
  block_sum<3>(part, red);
  if (threadIdx.x == 0) {
    A.part[blockIdx.x * 4 + 0] = part[0];
    A.part[blockIdx.x * 4 + 1] = part[1];
    A.part[blockIdx.x * 4 + 2] = part[2];
    __threadfence();
    const unsigned ticket = atomicAdd(&sc->counter, 1u);
    is_last = (ticket == (unsigned)sy.epi_blocks - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();

  double tot[3] = {0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < sy.epi_blocks; j += blockDim.x) {
    const int r = P.epipre[b] + j;
    tot[0] += __ldcg(&A.part[r * 4 + 0]);
    tot[1] += __ldcg(&A.part[r * 4 + 1]);
    tot[2] += __ldcg(&A.part[r * 4 + 2]);
  }
  block_sum<3>(tot, red);
  if (threadIdx.x == 0) {
    const double outflow = sc->gflux - tot[0];
    sc->outflow = outflow;
    switch (A.mode) {
      case EPI_RHS:
        if (A.outflow_out) A.outflow_out[b] = outflow;
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
          double* dr = A.diag + ((int64_t)row * P.B + b) * 3;
          dr[0] = tot[1];
          dr[1] = tot[2];
          dr[2] = sc->cum;
        }
        break;
      }
    }
    sc->counter = 0u;
    sc->nmax_bits = 0ull;
  }
}

// Row 0 of the diagnostics (M0, M1 of n, zero outflow) and the integrator's
// counters. One block per system.
__global__ void __launch_bounds__(1024) k_moments(const __grid_constant__ RhsParams P,
                                                  const double* __restrict__ n, double* diag) {
  __shared__ double red[64];
  const int b = blockIdx.x;
  const SysDesc sy = P.sys[b];
  const double* x = n + sy.noff;
  double acc[2] = {0.0, 0.0};
  for (int k = threadIdx.x; k < sy.N; k += blockDim.x) {
    acc[0] += x[k];
    acc[1] = fma((double)(k + 1), x[k], acc[1]);
  }
  block_sum<2>(acc, red);
  if (threadIdx.x == 0) {
    P.sc[b].step = 0;
    P.sc[b].cum = 0.0;
    if (diag) {
      diag[b * 3 + 0] = acc[0];
      diag[b * 3 + 1] = acc[1];
      diag[b * 3 + 2] = 0.0;
    }
  }
}

// ---- launch of one evaluation ---------------------------------------------
cudaError_t enqueue_eval(const RhsParams& P, const LaunchCfg& L, const double* nin,
                         const EpiArgs& A, cudaStream_t st, LaunchHook* hook, const SideStream* side,
                         const FftGroups* groups) {
  if (P.dwpath && !A.presplit) {
    if (hook) hook->mark(KID_NMAX, st);
    k_nmax<<<dim3(L.prep_blocks, P.B), 256, 0, st>>>(P, nin);
    if (hook) hook->mark(KID_NSPLIT, st);
    k_nsplit<<<dim3(L.prep_blocks, P.B), 256, 0, st>>>(P, nin);
  }
  // The inner products and loss weights (FP64 pipe) overlap the FFT kernels
  // (FP32 pipe) on the side stream; per-kernel timing runs everything in order.
  const bool fork = side != nullptr && hook == nullptr;
  cudaStream_t ds = fork ? side->stream : st;
  cudaError_t e;
  if (fork) {
    if ((e = cudaEventRecord(side->fork, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(ds, side->fork, 0)) != cudaSuccess) return e;
  }
  if (hook) hook->mark(KID_DOT, st);
  k_dot<<<dim3(P.Vtot, P.maxdotchunk), 256, 0, ds>>>(P, nin, A.flux);
  if (hook) hook->mark(KID_COEF, st);
  k_coef<<<P.B, 256, L.coef_smem, ds>>>(P, A.flux);
  if (hook) hook->mark(KID_QTERM, st);
  k_qterm<<<L.epi_blocks, 256, L.epi_smem, ds>>>(P, nin);
  if (fork && (e = cudaEventRecord(side->join, ds)) != cudaSuccess) return e;
  if (fork && groups && groups->n > 1) {
    // one FFT chain per group, each on its own stream after the split of n
    for (int g = 0; g < groups->n; ++g) {
      cudaStream_t gs = groups->s[g].stream;
      if ((e = cudaStreamWaitEvent(gs, side->fork, 0)) != cudaSuccess) return e;
      e = P.dwpath ? enqueue_fft_dw(P, L, nin, gs, nullptr, &groups->r[g])
                   : enqueue_fft_f64(P, L, nin, gs, nullptr, &groups->r[g]);
      if (e != cudaSuccess) return e;
      if ((e = cudaEventRecord(groups->s[g].join, gs)) != cudaSuccess) return e;
    }
    for (int g = 0; g < groups->n; ++g)
      if ((e = cudaStreamWaitEvent(st, groups->s[g].join, 0)) != cudaSuccess) return e;
  } else {
    e = P.dwpath ? enqueue_fft_dw(P, L, nin, st, hook) : enqueue_fft_f64(P, L, nin, st, hook);
    if (e != cudaSuccess) return e;
  }
  if (fork && (e = cudaStreamWaitEvent(st, side->join, 0)) != cudaSuccess) return e;
  if (hook) hook->mark(KID_EPILOGUE, st);
  k_epilogue<<<L.epi_blocks, 256, 0, st>>>(P, A);
  if (hook) hook->mark(-1, st);
  return cudaGetLastError();
}

cudaError_t enqueue_nsplit(const RhsParams& P, const LaunchCfg& L, const double* n, cudaStream_t st) {
  k_nmax<<<dim3(L.prep_blocks, P.B), 256, 0, st>>>(P, n);
  k_nsplit<<<dim3(L.prep_blocks, P.B), 256, 0, st>>>(P, n);
  return cudaGetLastError();
}

cudaError_t enqueue_moments(const RhsParams& P, const double* n, double* diag, cudaStream_t st) {
  k_moments<<<P.B, 1024, 0, st>>>(P, n, diag);
  return cudaGetLastError();
}

cudaError_t setup_common_kernels(const LaunchCfg& L) {
  cudaError_t e = allow_max_smem(k_qterm);
  if (e == cudaSuccess)
    e = allow_max_smem(k_coef);
  return e;
}

// ---- one RK2 stage from a given right-hand side k (the term-parallel split,
// where k is the sum of the ranks' partial right-hand sides): stage 0 stores
// k1 = k and the intermediate state nstar = n + h1 k (h1 = dt for Heun, dt/2
// for the midpoint rule); stage 1 advances n by dt/2 (k1 + k) (Heun) or
// dt k (midpoint). A non-finite k latches the plan's status.
__global__ void k_rk2_stage(const __grid_constant__ RhsParams P, int stage, int midpoint, double* n,
                            double* nstar, double* k1, const double* __restrict__ k, double dt) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.Ntot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ki = k[i];
    bad |= !isfinite(ki);
    if (stage == 0) {
      k1[i] = ki;
      nstar[i] = n[i] + (midpoint ? 0.5 * dt : dt) * ki;
    } else {
      n[i] = midpoint ? n[i] + dt * ki : n[i] + 0.5 * dt * (k1[i] + ki);
    }
  }
  if (bad) atomicOr(P.status, kStatusNonFinite);
}

cudaError_t enqueue_rk2_stage(const RhsParams& P, int stage, int midpoint, double* n, double* nstar,
                              double* k1, const double* k, double dt, cudaStream_t st) {
  const int64_t want = (P.Ntot + 255) / 256;
  const int blocks = (int)(want < 4096 ? want : 4096);
  k_rk2_stage<<<blocks, 256, 0, st>>>(P, stage, midpoint, n, nstar, k1, k, dt);
  return cudaGetLastError();
}

// ---- the parametric factors' generator on its own: out[i - 1] = u i^a for
// i = 1..N, evaluated exactly as the forward column kernels do (dw_pow.cuh)
// and returned as hi + lo in FP64.
__global__ void k_power_eval(float4 up, const float2* __restrict__ lnt, const float* __restrict__ ek, int N,
                             double* __restrict__ out) {
  for (int i = 1 + blockIdx.x * blockDim.x + threadIdx.x; i <= N; i += gridDim.x * blockDim.x) {
    const float2 l = lnt[i];
    const dw y = dw_power(dw{up.x, up.y}, dw{up.z, up.w}, dw{l.x, l.y}, ek);
    out[i - 1] = (double)y.hi + (double)y.lo;
  }
}

cudaError_t enqueue_power_eval(float4 up, const float2* lnt, const float* ek, int N, double* out, cudaStream_t st) {
  const int blocks = (N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096;
  k_power_eval<<<blocks, 256, 0, st>>>(up, lnt, ek, N, out);
  return cudaGetLastError();
}

}  // namespace sag
