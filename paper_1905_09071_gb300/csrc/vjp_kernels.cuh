// Vector-Jacobian product of the CP right-hand side (the adjoint used for
// kernel fitting), templated on the complex scalar.
//
// For the gain term, p_k = 1/d! sum_r (a^(1)_r * ... * a^(d)_r)[k] with
// a^(m)_r = U^(m)_r o n, the cotangent of a^(m)_r is
//   ga^(m)_r[i] = 1/d! sum_k g_k (conv_{m' != m} a^(m')_r)[k - i],
// a correlation: in the frequency domain G[w] conj(prod_{m' != m} A^(m')_r[w]),
// inverse-transformed at the same length L >= d N as the forward pass (the
// correlation outputs 1..N do not alias). Per row pair of the four-step
// transform the kernel computes the forward rows of g and of the d vectors
// of each rank term, forms the d products with prefix/suffix products
// (no division), and runs the inverse row half for each of them; the inverse
// column kernel then writes ga per vector.
#pragma once

#include "fft_kernels.cuh"

namespace sag {

// ---- g: column pass of each item's cotangent (sizes 1..N, as a real sequence)
__device__ __forceinline__ cd load_pair_raw(const double* __restrict__ x, int N, int k, cd) {
  return cd{(k >= 1 && k <= N) ? x[k - 1] : 0.0, (k + 1 <= N) ? x[k] : 0.0};
}
__device__ __forceinline__ cdw load_pair_raw(const float2* __restrict__ x, int N, int k, cdw) {
  dw re{0.f, 0.f}, im{0.f, 0.f};
  if (k >= 1 && k <= N) re = dw{x[k - 1].x, x[k - 1].y};
  if (k + 1 <= N) im = dw{x[k].x, x[k].y};
  return make_cdw(re, im);
}
__device__ __forceinline__ const double* g_ptr(const RhsParams&, const double* g, int64_t off, cd) {
  return g + off;
}
__device__ __forceinline__ const float2* g_ptr(const RhsParams& P, const double*, int64_t off, cdw) {
  return P.gdw + off;
}

template <class C>
__global__ void __launch_bounds__(kThreads) k_gcol(const __grid_constant__ RhsParams P,
                                                   const double* __restrict__ g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int it = find_segment(P.invpre, P.nitems, blockIdx.x);
  const OrderDesc& od = P.ord[it];
  const int cb = blockIdx.x - P.invpre[it];
  const int W = od.W, M1 = od.M1, M2 = od.M2, ld = od.ld1, N = od.N;
  C* buf1 = buf + W * ld;
  C* tw = buf1 + W * ld;
  const C* tw1 = static_cast<const C*>(od.tw1);
  for (int i = threadIdx.x; i < M1; i += kThreads) tw[i] = tw1[i];
  const auto x = g_ptr(P, g, od.noff, C{});
  for (int e = threadIdx.x; e < W * M1; e += kThreads) {
    const int c = e % W, j1 = e / W;
    buf[c * ld + j1] = load_pair_raw(x, N, 2 * (M2 * j1 + cb * W + c), C{});
  }
  __syncthreads();
  C* res = fft_batch(buf, buf1, M1, ld, W, od.rp1, tw);
  C* dst = static_cast<C*>(P.scratch2) + od.scr2_off;
  const C* tw4 = static_cast<const C*>(od.tw4);
  for (int e = threadIdx.x; e < W * M1; e += kThreads) {
    const int c = e % W, k1 = e / W, j2 = cb * W + c;
    dst[(int64_t)k1 * M2 + j2] = c_mul(res[c * ld + k1], tw4[j2 * k1]);
  }
}

// ---- row pass of the product rule ------------------------------------------
template <class C>
__global__ void __launch_bounds__(kThreads) k_rows_vjp(const __grid_constant__ RhsParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int j = find_segment(P.rowpre, P.nitems, blockIdx.x);
  const OrderDesc& od = P.ord[P.rowperm[j]];
  const int kp = blockIdx.x - P.rowpre[j];
  const int d = od.d, R = od.R, M1 = od.M1, M2 = od.M2, M = od.M, ld = od.ld2;
  // One block per (row pair, rank term r = blockIdx.y): the terms' vectors
  // have slots of their own, and each block forms g's row spectrum again.
  const int r = blockIdx.y;
  if (r >= R) return;
  const int k1a = kp, k1b = M1 - kp;
  const int nrow = (kp == 0 || 2 * kp == M1) ? 1 : 2;
  const int NP = nrow * M2;
  const int NS = 2 * M2 + 1;  // spectrum slots per vector (positions and the Nyquist value)
  // With RhsParams::vjp_gmerge, g's rows are transformed in the same batch as
  // the term's d vectors (slot 0, one load and one transform phase fewer);
  // the plan sets it when the d + 1 slots fit the shared memory.
  const int gm = P.vjp_gmerge, nb = d + gm;
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + nb * 2 * ld;
  C* Gs = buf1 + nb * 2 * ld;
  C* A = Gs + NS;  // Gs and the d spectra A_m, NS apart
  C* tw = A + d * NS;
  const C* tw2 = static_cast<const C*>(od.tw2);
  const C* twL = static_cast<const C*>(od.twL);
  const C* tw4 = static_cast<const C*>(od.tw4);
  C* vec = static_cast<C*>(P.scratch) + od.scr_off;
  const C* gsrc = static_cast<const C*>(P.scratch2) + od.scr2_off;
  const bool nyq = kp == 0;
  for (int i = threadIdx.x; i < M2; i += kThreads) tw[i] = tw2[i];
  C* res;
  if (!gm) {
    // Spectrum of g at the block's positions.
    for (int p = threadIdx.x; p < NP; p += kThreads) {
      const int row = p / M2, pos = p - row * M2;
      buf0[row * ld + pos] = gsrc[(int64_t)(row ? k1b : k1a) * M2 + pos];
    }
    __syncthreads();
    res = fft_batch(buf0, buf1, M2, ld, nrow, od.rp2, tw);
    for (int p = threadIdx.x; p < NP; p += kThreads) {
      const int row = p / M2, pos = p - row * M2;
      const int k1 = row ? k1b : k1a;
      int mrow, mpos;
      mirror_of(k1, row, pos, M1, M2, mrow, mpos);
      Gs[p] = unpack2(res[row * ld + pos], res[mrow * ld + mpos], twL[k1 + M1 * pos]);
    }
    if (nyq && threadIdx.x == 0) {
      const C z0 = res[0];
      const C zc = c_conj(z0);
      Gs[NP] = c_add(c_add(z0, zc), c_mul_pi(c_sub(z0, zc)));
    }
    __syncthreads();
  }

  {
    // forward rows of the d vectors of rank term r (after g's, slot 0, when merged)
    for (int e = threadIdx.x; e < nb * NP; e += kThreads) {
      const int m = e / NP, p = e - m * NP;
      const int row = p / M2, pos = p - row * M2;
      const int k1 = row ? k1b : k1a;
      buf0[(m * nrow + row) * ld + pos] =
          (gm && m == 0) ? gsrc[(int64_t)k1 * M2 + pos] : vec[(int64_t)((m - gm) * R + r) * M + (int64_t)k1 * M2 + pos];
    }
    __syncthreads();
    res = fft_batch(buf0, buf1, M2, ld, nb * nrow, od.rp2, tw);
    C* Sp = gm ? Gs : A;  // spectrum m of the batch goes to Sp + m NS
    for (int e = threadIdx.x; e < nb * NP; e += kThreads) {
      const int m = e / NP, p = e - m * NP;
      const int row = p / M2, pos = p - row * M2;
      const int k1 = row ? k1b : k1a;
      int mrow, mpos;
      mirror_of(k1, row, pos, M1, M2, mrow, mpos);
      Sp[m * NS + p] = unpack2(res[(m * nrow + row) * ld + pos], res[(m * nrow + mrow) * ld + mpos],
                               twL[k1 + M1 * pos]);
    }
    if (nyq && threadIdx.x < nb) {
      const int m = threadIdx.x;
      const C z0 = res[(m * nrow) * ld];
      const C zc = c_conj(z0);
      Sp[m * NS + NP] = c_add(c_add(z0, zc), c_mul_pi(c_sub(z0, zc)));
    }
    __syncthreads();
    // H_m = G conj(prod_{m' != m} A_m'), by prefix and suffix products
    for (int p = threadIdx.x; p < NP + (nyq ? 1 : 0); p += kThreads) {
      C pre[kMaxD];
      C acc = c_one(C{});
#pragma unroll
      for (int m = 0; m < kMaxD; ++m) {
        if (m < d) {
          pre[m] = acc;
          acc = c_mul(acc, c_conj(A[m * NS + p]));
        }
      }
      C suf = Gs[p];
#pragma unroll
      for (int m = kMaxD - 1; m >= 0; --m) {
        if (m < d) {
          const C am = c_conj(A[m * NS + p]);
          A[m * NS + p] = c_mul(pre[m], suf);
          suf = c_mul(suf, am);
        }
      }
    }
    __syncthreads();
    // inverse row half of each H_m (as in the forward inverse)
    for (int e = threadIdx.x; e < d * NP; e += kThreads) {
      const int m = e / NP, p = e - m * NP;
      const int row = p / M2, pos = p - row * M2;
      const int k1 = row ? k1b : k1a;
      const int k = k1 + M1 * pos;
      int mrow, mpos;
      mirror_of(k1, row, pos, M1, M2, mrow, mpos);
      const C Sk = A[m * NS + p];
      const C Sm = (k == 0) ? A[m * NS + NP] : c_conj(A[m * NS + mrow * M2 + mpos]);
      const C zpp = c_add(c_add(Sk, Sm), c_mul_pi(c_mul(c_conj(twL[k]), c_sub(Sk, Sm))));
      buf0[(m * nrow + row) * ld + pos] = c_conj(zpp);
    }
    __syncthreads();
    res = fft_batch(buf0, buf1, M2, ld, d * nrow, od.rp2, tw);
    for (int e = threadIdx.x; e < d * NP; e += kThreads) {
      const int m = e / NP, p = e - m * NP;
      const int row = p / M2, j2 = p - row * M2;
      const int k1 = row ? k1b : k1a;
      vec[(int64_t)(m * R + r) * M + (int64_t)k1 * M2 + j2] =
          c_mul(res[(m * nrow + row) * ld + j2], tw4[j2 * k1]);
    }
    __syncthreads();
  }
}

// ---- inverse column pass per vector: the cotangent ga of a = U o n ---------
template <class C>
__global__ void __launch_bounds__(kThreads) k_inv_col_vjp(const __grid_constant__ RhsParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int it = find_segment(P.colpre_all, P.nitems, blockIdx.x);
  const OrderDesc& od = P.ord[it];
  const int local = blockIdx.x - P.colpre_all[it];
  const int vloc = local / od.ncolblk, cb = local - vloc * od.ncolblk;
  const int v = od.vbase + vloc;
  const int W = od.W, M1 = od.M1, M2 = od.M2, ld = od.ld1, N = od.N;
  C* buf1 = buf + W * ld;
  C* tw = buf1 + W * ld;
  const C* tw1 = static_cast<const C*>(od.tw1);
  for (int i = threadIdx.x; i < M1; i += kThreads) tw[i] = tw1[i];
  const C* src = static_cast<const C*>(P.scratch) + od.scr_off + (int64_t)vloc * od.M;
  for (int e = threadIdx.x; e < W * M1; e += kThreads) {
    const int c = e % W, k1 = e / W;
    buf[c * ld + k1] = src[(int64_t)k1 * M2 + cb * W + c];
  }
  __syncthreads();
  C* res = fft_batch(buf, buf1, M1, ld, W, od.rp1, tw);
  const SysScalars& sc = P.sc[od.sys];
  const int ex = P.dwpath ? sc.e_g + P.vexcl[v] + (od.d - 1) * sc.e_n : 0;
  const double scale = ldexp(od.gscale, ex);
  double* out = P.gabuf + P.voff[v];
  for (int e = threadIdx.x; e < W * M1; e += kThreads) {
    const int c = e % W, j1 = e / W;
    const int jj = M2 * j1 + cb * W + c;
    const C w = res[c * ld + j1];
    const int k = 2 * jj;
    if (k >= 1 && k <= N) out[k - 1] = cre(w) * scale;
    if (k + 1 <= N) out[k] = -cim(w) * scale;
  }
}

}  // namespace sag
