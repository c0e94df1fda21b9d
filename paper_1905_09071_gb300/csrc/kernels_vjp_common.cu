// Vector-Jacobian product of the CP right-hand side: the non-FFT kernels
// (cotangent scaling, inner products, loss-term derivatives, assembly) and
// the launch sequence. The loss term q_k = n_k sum_v coef_v U_v(k), with
// coef_v built from the inner products s = <U, n>, is differentiated by the
// product rule: through n_k, through U_v(k), and through every s in coef:
//   sigma_v = dL/ds_v = sum_{v' of the same rank term, v' != v}
//             z_{v'} d coef_{v'} / d s_v,   z_v = <U_v, g o n>.
#include "launch.h"

namespace sag {

cudaError_t launch_vjp_fft_dw(const RhsParams& P, const LaunchCfg& L, const double* n, const double* g,
                              cudaStream_t st);
cudaError_t launch_vjp_fft_f64(const RhsParams& P, const LaunchCfg& L, const double* n, const double* g,
                               cudaStream_t st);
cudaError_t launch_vjp_fft_tt_dw(const RhsParams& P, const LaunchCfg& L, const double* n, const double* g,
                                 cudaStream_t st);
cudaError_t launch_vjp_fft_tt_f64(const RhsParams& P, const LaunchCfg& L, const double* n, const double* g,
                                  cudaStream_t st);

namespace {

template <int NV>
__device__ __forceinline__ void block_sum_v(double (&v)[NV], double* sh) {
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

__device__ __forceinline__ double inv_fact(int d) {
  double f = 1.0;
  for (int i = 2; i <= d; ++i) f *= i;
  return 1.0 / f;
}

// g for the double-word path: g 2^-e_g with max |g| 2^-e_g in [0.5, 1), per system.
__global__ void k_gmax(const __grid_constant__ RhsParams P, const double* __restrict__ g) {
  const SysDesc s = P.sys[blockIdx.y];
  const double* x = g + s.noff;
  double m = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < s.N; k += gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[k]));
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0)
    atomicMax(&P.sc[blockIdx.y].gmax_bits, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_gsplit(const __grid_constant__ RhsParams P, const double* __restrict__ g) {
  const SysDesc s = P.sys[blockIdx.y];
  SysScalars* sc = &P.sc[blockIdx.y];
  const double mx = __longlong_as_double((long long)sc->gmax_bits);
  const int e = (mx > 0.0 && isfinite(mx)) ? ilogb(mx) + 1 : 0;
  const double* x = g + s.noff;
  float2* out = P.gdw + s.noff;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < s.N; k += gridDim.x * blockDim.x) {
    const dw v = dw_from_double(scalbn(x[k], -e));
    out[k] = make_float2(v.hi, v.lo);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->e_g = e;
}

// s_v = <U_v, n> and z_v = <U_v, g o n> partial sums (FP64).
__global__ void __launch_bounds__(256) k_dot2(const __grid_constant__ RhsParams P,
                                              const double* __restrict__ n,
                                              const double* __restrict__ g) {
  __shared__ double sh[64];
  const int v = blockIdx.x, c = blockIdx.y;
  const SysDesc s = P.sys[P.vsys[v]];
  if (c >= s.ndotchunk) return;
  const int k0 = c * P.dotchunk, k1 = min(s.N, k0 + P.dotchunk);
  const double* u = P.U64 + P.voff[v];
  const double* x = n + s.noff;
  const double* y = g + s.noff;
  double acc[2] = {0.0, 0.0};
  for (int k = k0 + threadIdx.x; k < k1; k += 256) {
    const double un = u[k] * x[k];
    acc[0] += un;
    acc[1] = fma(un, y[k], acc[1]);
  }
  block_sum_v<2>(acc, sh);
  if (threadIdx.x == 0) {
    P.dot_s[(int64_t)v * P.maxdotchunk + c] = acc[0];
    P.dot_z[(int64_t)v * P.maxdotchunk + c] = acc[1];
  }
}

// coef_v (as in the forward pass) and sigma_v, one block per system.
__global__ void __launch_bounds__(256) k_coef_vjp(const __grid_constant__ RhsParams P) {
  extern __shared__ double csh[];  // s, z of the system's vectors
  const int b = blockIdx.x;
  const SysDesc sy = P.sys[b];
  const int nv = sy.vend - sy.vbeg, nc = sy.ndotchunk;
  double* s = csh;
  double* z = csh + nv;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const int64_t base = (int64_t)(sy.vbeg + i) * P.maxdotchunk;
    double a = 0.0, c2 = 0.0;
    for (int c = 0; c < nc; ++c) {
      a += P.dot_s[base + c];
      c2 += P.dot_z[base + c];
    }
    s[i] = a;
    z[i] = c2;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const int v = sy.vbeg + i;
    int it = sy.ibeg;
    while (it + 1 < sy.iend && v >= P.ord[it + 1].vbase) ++it;
    const OrderDesc& od = P.ord[it];
    const int d = od.d, R = od.R, loc = v - od.vbase, m = loc / R, r = loc - m * R;
    const int lb = od.vbase - sy.vbeg;
    const double f1 = inv_fact(d - 1);
    double prod = 1.0;
    for (int mm = 0; mm < d; ++mm)
      if (mm != m) prod *= s[lb + mm * R + r];
    const double wm = P.sym ? 1.0 / d : (m == d - 1 ? 1.0 : 0.0);
    P.coef[v] = -f1 * wm * prod;
    double sg = 0.0;
    for (int m2 = 0; m2 < d; ++m2) {
      if (m2 == m) continue;
      const double w2 = P.sym ? 1.0 / d : (m2 == d - 1 ? 1.0 : 0.0);
      double p2 = -f1 * w2 * z[lb + m2 * R + r];
      for (int mm = 0; mm < d; ++mm)
        if (mm != m2 && mm != m) p2 *= s[lb + mm * R + r];
      sg += p2;
    }
    P.sigma[v] = sg;
  }
  if (threadIdx.x == 0) {
    P.sc[b].nmax_bits = 0ull;
    P.sc[b].gmax_bits = 0ull;
  }
}

// ---- TT: coef and sigma of every core entry, one block per order ----------
// M_l[a][b] = <h^(l)_{a,b}, n>, Z_l[a][b] = <h^(l)_{a,b}, g o n> (0 for
// entries without a vector). Entry (l, a, b): coef = c w_l left[a] right[b]
// of the M chain, sigma = c sum_{pos != l} w_pos pre[a] suf[b] of the chain
// with Z_pos in place of M_pos, c = -1/(d-1)!, w = 1/d (symmetrised) or
// [pos = d] (last mode).
constexpr int kTR = kMaxTTRank;
__device__ void tt_left(const double* Mx, const double* Zx, int zpos, const int* ttr, int upto, double* out) {
  // out = e_0^T X_1 ... X_upto, X_l = Z_l if l == zpos else M_l
  double tmp[kTR];
  out[0] = 1.0;
  for (int l = 1; l <= upto; ++l) {
    const double* X = (l == zpos ? Zx : Mx) + (l - 1) * kTR * kTR;
    for (int b = 0; b < ttr[l]; ++b) {
      double acc = 0.0;
      for (int a = 0; a < ttr[l - 1]; ++a) acc = fma(out[a], X[a * kTR + b], acc);
      tmp[b] = acc;
    }
    for (int b = 0; b < ttr[l]; ++b) out[b] = tmp[b];
  }
}
__device__ void tt_right(const double* Mx, const double* Zx, int zpos, const int* ttr, int d, int from,
                         double* out) {
  // out = X_from ... X_d e_0
  double tmp[kTR];
  out[0] = 1.0;
  for (int l = d; l >= from; --l) {
    const double* X = (l == zpos ? Zx : Mx) + (l - 1) * kTR * kTR;
    for (int a = 0; a < ttr[l - 1]; ++a) {
      double acc = 0.0;
      for (int b = 0; b < ttr[l]; ++b) acc = fma(X[a * kTR + b], out[b], acc);
      tmp[a] = acc;
    }
    for (int a = 0; a < ttr[l - 1]; ++a) out[a] = tmp[a];
  }
}

__global__ void __launch_bounds__(256) k_coef_vjp_tt(const __grid_constant__ RhsParams P) {
  __shared__ double Mx[kMaxD * kTR * kTR], Zx[kMaxD * kTR * kTR];
  const int it = blockIdx.x;
  const OrderDesc& od = P.ord[it];
  const SysDesc sy = P.sys[od.sys];
  const int d = od.d, nc = sy.ndotchunk;
  const int* vid = P.vid + od.vid_off;
  for (int q = threadIdx.x; q < od.nent; q += blockDim.x) {
    int l = 1, off = 0;
    while (q >= off + od.ttr[l - 1] * od.ttr[l]) off += od.ttr[l - 1] * od.ttr[l++];
    const int loc = q - off, a = loc / od.ttr[l], b = loc - a * od.ttr[l];
    const int v = vid[q];
    double sm = 0.0, sz = 0.0;
    if (v >= 0) {
      const int64_t base = (int64_t)v * P.maxdotchunk;
      for (int c = 0; c < nc; ++c) {
        sm += P.dot_s[base + c];
        sz += P.dot_z[base + c];
      }
    }
    Mx[(l - 1) * kTR * kTR + a * kTR + b] = sm;
    Zx[(l - 1) * kTR * kTR + a * kTR + b] = sz;
  }
  __syncthreads();
  const double c = -inv_fact(d - 1);
  for (int q = threadIdx.x; q < od.nent; q += blockDim.x) {
    int l = 1, off = 0;
    while (q >= off + od.ttr[l - 1] * od.ttr[l]) off += od.ttr[l - 1] * od.ttr[l++];
    const int loc = q - off, a = loc / od.ttr[l], b = loc - a * od.ttr[l];
    double left[kTR], right[kTR];
    const double wl = P.sym ? 1.0 / d : (l == d ? 1.0 : 0.0);
    double coef = 0.0;
    if (wl != 0.0) {
      tt_left(Mx, Zx, 0, od.ttr, l - 1, left);
      tt_right(Mx, Zx, 0, od.ttr, d, l + 1, right);
      coef = c * wl * left[a] * right[b];
    }
    double sg = 0.0;
    for (int pos = 1; pos <= d; ++pos) {
      if (pos == l) continue;
      const double wp = P.sym ? 1.0 / d : (pos == d ? 1.0 : 0.0);
      if (wp == 0.0) continue;
      tt_left(Mx, Zx, pos, od.ttr, l - 1, left);
      tt_right(Mx, Zx, pos, od.ttr, d, l + 1, right);
      sg += c * wp * left[a] * right[b];
    }
    P.coef[od.ebase + q] = coef;
    P.sigma[od.ebase + q] = sg;
  }
  if (threadIdx.x == 0 && it == sy.ibeg) {
    P.sc[od.sys].nmax_bits = 0ull;
    P.sc[od.sys].gmax_bits = 0ull;
  }
}

// gn_k = g_k sum_e coef_e h_e(k) + sum_e h_e(k) (ga_e(k) + sigma_e),
// gH_e(k) (=|+=) n_k (ga_e(k) + sigma_e) + coef_e g_k n_k, over every core
// entry of the system (h_e = 0 for an entry without a stored vector).
__global__ void __launch_bounds__(256) k_vjp_final_tt(const __grid_constant__ RhsParams P,
                                                      const double* __restrict__ n,
                                                      const double* __restrict__ g, double* gn,
                                                      double* gH, int accumulate) {
  const int b = find_segment(P.epipre, P.B, blockIdx.x);
  const SysDesc sy = P.sys[b];
  const int k = (blockIdx.x - P.epipre[b]) * blockDim.x + threadIdx.x;
  if (k >= sy.N) return;
  const int64_t gk = sy.noff + k;
  const double nk = n[gk], gg = g[gk];
  double w = 0.0, acc = 0.0;
  for (int it = sy.ibeg; it < sy.iend; ++it) {
    const OrderDesc& od = P.ord[it];
    const int* vid = P.vid + od.vid_off;
    for (int q = 0; q < od.nent; ++q) {
      const int e = od.ebase + q, v = vid[q];
      const double h = v >= 0 ? P.U64[P.voff[v] + k] : 0.0;
      const int64_t o = P.eoff[e] + k;
      const double ga = P.gaent[o] + P.sigma[e];
      const double cf = P.coef[e];
      w = fma(cf, h, w);
      acc = fma(h, ga, acc);
      if (gH) {
        const double val = fma(nk, ga, cf * gg * nk);
        gH[o] = accumulate ? gH[o] + val : val;
      }
    }
  }
  if (gn) gn[gk] = fma(gg, w, acc);
}

// gn_k = g_k w_k + sum_v U_v(k) (ga_v(k) + sigma_v),
// gU_v(k) (=|+=) n_k (ga_v(k) + sigma_v) + coef_v g_k n_k.
// Each 256-size epilogue block splits into kFinSplit blocks of 32 sizes x 8
// vector groups (a warp: 32 consecutive sizes of one group, every eighth
// vector); group 0 adds the other groups' partial sums in a fixed order.
constexpr int kFinSizes = 32, kFinGroups = 8, kFinSplit = 256 / kFinSizes;
__global__ void __launch_bounds__(256) k_vjp_final(const __grid_constant__ RhsParams P,
                                                   const double* __restrict__ n,
                                                   const double* __restrict__ g, double* gn,
                                                   double* gU, int accumulate) {
  extern __shared__ double fsh[];  // coef, sigma of the system's vectors
  __shared__ double part[kFinGroups - 1][2][kFinSizes];
  const int eb = blockIdx.x / kFinSplit, sub = blockIdx.x - eb * kFinSplit;
  const int b = find_segment(P.epipre, P.B, eb);
  const SysDesc sy = P.sys[b];
  const int nv = sy.vend - sy.vbeg, N = sy.N;
  const int kbase = (eb - P.epipre[b]) * 256 + sub * kFinSizes;
  if (kbase >= N) return;  // the whole block
  double* coef = fsh;
  double* sig = fsh + nv;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    coef[i] = P.coef[sy.vbeg + i];
    sig[i] = P.sigma[sy.vbeg + i];
  }
  __syncthreads();
  const int kl = threadIdx.x % kFinSizes, grp = threadIdx.x / kFinSizes;
  const int k = kbase + kl;
  double w = 0.0, acc = 0.0;
  if (k < N) {
    const int64_t gk = sy.noff + k;
    const double nk = n[gk], gg = g[gk];
    const int64_t base = P.voff[sy.vbeg] + k;  // a system's vectors are stored back to back
    for (int i = grp; i < nv; i += kFinGroups) {
      const int64_t o = base + (int64_t)i * N;
      const double u = P.U64[o];
      const double ga = P.gabuf[o] + sig[i];
      w = fma(coef[i], u, w);
      acc = fma(u, ga, acc);
      if (gU) {
        const double val = fma(nk, ga, coef[i] * gg * nk);
        gU[o] = accumulate ? gU[o] + val : val;
      }
    }
  }
  if (grp > 0) {
    part[grp - 1][0][kl] = w;
    part[grp - 1][1][kl] = acc;
  }
  __syncthreads();
  if (grp > 0 || k >= N) return;
  for (int q = 0; q < kFinGroups - 1; ++q) {
    w += part[q][0][kl];
    acc += part[q][1][kl];
  }
  const int64_t gk = sy.noff + k;
  if (gn) gn[gk] = fma(g[gk], w, acc);
}

__global__ void k_axpby(double* out, double a, const double* x, double b, const double* y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (y ? fma(a, x[i], b * y[i]) : a * x[i]);
}

}  // namespace

cudaError_t enqueue_vjp(const RhsParams& P, const LaunchCfg& L, const double* n, const double* g,
                        double* gn, double* gU, int accumulate, cudaStream_t st, const SideStream* side) {
  cudaError_t e;
  if (P.dwpath) {
    // n and g to double-word with their own power-of-two scales; the max
    // counters start at zero and k_coef_vjp resets them for the next call.
    enqueue_nsplit(P, L, n, st);
    k_gmax<<<dim3(L.prep_blocks, P.B), 256, 0, st>>>(P, g);
    k_gsplit<<<dim3(L.prep_blocks, P.B), 256, 0, st>>>(P, g);
  }
  // The inner products and weights of the product rule need only n and g:
  // on the side stream, beside the FFT kernels, from here on (after the
  // splits, whose max counters k_coef_vjp clears); the final kernel joins.
  cudaStream_t ds = side ? side->stream : st;
  if (side) {
    if ((e = cudaEventRecord(side->fork, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(ds, side->fork, 0)) != cudaSuccess) return e;
  }
  k_dot2<<<dim3(P.Vtot, P.maxdotchunk), 256, 0, ds>>>(P, n, g);
  if (L.has_tt) k_coef_vjp_tt<<<P.nitems, 256, 0, ds>>>(P);
  else k_coef_vjp<<<P.B, 256, L.coef_smem, ds>>>(P);
  if (side && (e = cudaEventRecord(side->join, ds)) != cudaSuccess) return e;
  if (L.has_tt) e = P.dwpath ? launch_vjp_fft_tt_dw(P, L, n, g, st) : launch_vjp_fft_tt_f64(P, L, n, g, st);
  else e = P.dwpath ? launch_vjp_fft_dw(P, L, n, g, st) : launch_vjp_fft_f64(P, L, n, g, st);
  if (e != cudaSuccess) return e;
  if (side && (e = cudaStreamWaitEvent(st, side->join, 0)) != cudaSuccess) return e;
  if (L.has_tt) k_vjp_final_tt<<<L.epi_blocks, 256, 0, st>>>(P, n, g, gn, gU, accumulate);
  else k_vjp_final<<<L.epi_blocks * kFinSplit, 256, L.coef_smem, st>>>(P, n, g, gn, gU, accumulate);
  return cudaGetLastError();
}

cudaError_t enqueue_axpby(double* out, double a, const double* x, double b, const double* y, int64_t n,
                          cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  k_axpby<<<blocks, 256, 0, st>>>(out, a, x, b, y, n);
  return cudaGetLastError();
}

cudaError_t setup_vjp_common(const LaunchCfg& L) {
  (void)L;
  cudaError_t e = allow_max_smem(k_coef_vjp);
  if (e == cudaSuccess)
    e = allow_max_smem(k_vjp_final);
  return e;
}

}  // namespace sag
