// The three FFT kernels of one right-hand-side evaluation, templated on the
// complex scalar (cd: FP64; cdw: double-word FP32). For every order d:
//
//   k_fwd_col : a^(m)_r = U^(m)_r o n (Sec. 1, the vectors whose d-fold
//               convolution forms the gain term) packed two sizes per complex
//               point, column FFTs of the four-step transform, twiddle, store.
//   k_rows    : row FFTs of every vector, split into the real spectra A[k],
//               product over the d modes and sum over the ranks
//               S_d[k] = sum_r prod_m A^(m)_r[k] (convolution theorem), then
//               the first (row) half of the inverse transform of S_d.
//   k_inv_col : column half of the inverse; keeps sizes 1..N, scales by
//               1/d! and writes P^(d).
//
// Index conventions (see OrderDesc): real index = size, complex point
// j = M2 j1 + j2 holds sizes 2j and 2j+1; spectrum index k = k1 + M1 k2.
#pragma once

#include "plan.h"

namespace sag {

// ---- loading a = U o n, two sizes per complex point -------------------------
__device__ __forceinline__ cd load_a_pair(const RhsParams& P, int v, int k, const double* n, cd) {
  double re = 0.0, im = 0.0;
  const double* u = P.U64 + (int64_t)v * P.N;
  if (k >= 1 && k <= P.N) re = u[k - 1] * n[k - 1];
  if (k + 1 <= P.N) im = u[k] * n[k];
  return cd{re, im};
}
__device__ __forceinline__ cdw load_a_pair(const RhsParams& P, int v, int k, const double*, cdw) {
  dw re{0.f, 0.f}, im{0.f, 0.f};
  const float2* u = P.Udw + (int64_t)v * P.N;
  if (k >= 1 && k <= P.N) {
    float2 a = u[k - 1], b = P.ndw[k - 1];
    re = dw_mul(dw{a.x, a.y}, dw{b.x, b.y});
  }
  if (k + 1 <= P.N) {
    float2 a = u[k], b = P.ndw[k];
    im = dw_mul(dw{a.x, a.y}, dw{b.x, b.y});
  }
  return make_cdw(re, im);
}

// Power-of-two weight of a rank term (double-word path keeps every factor
// vector scaled to max |U| in [0.5, 1)); the FP64 path needs none.
__device__ __forceinline__ cd rank_weight(cd x, const OrderDesc&, int) { return x; }
__device__ __forceinline__ cdw rank_weight(cdw x, const OrderDesc& od, int r) {
  return c_scale2(x, od.rscale[r]);
}

// Twice the spectrum of a real sequence from its half-length packed transform:
// 2 A[k] = (Z[k] + conj Z[M-k]) - i omega_L^k (Z[k] - conj Z[M-k]).
template <class C>
__device__ __forceinline__ C unpack2(C zk, C zm, C wL) {
  C zc = c_conj(zm);
  return c_sub(c_add(zk, zc), c_mul_pi(c_mul(wL, c_sub(zk, zc))));
}

__device__ __forceinline__ int find_order(const int* pre, int nord, int b) {
  int oi = 0;
  while (oi + 1 < nord && b >= pre[oi + 1]) ++oi;
  return oi;
}

// ---------------------------------------------------------------------------
template <class C>
__global__ void __launch_bounds__(kThreads) k_fwd_col(const __grid_constant__ RhsParams P,
                                                      const double* __restrict__ n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int oi = find_order(P.colpre, P.nord, blockIdx.x);
  const OrderDesc& od = P.ord[oi];
  const int local = blockIdx.x - P.colpre[oi];
  const int vloc = local / od.ncolblk, cb = local - vloc * od.ncolblk;
  const int v = od.vbase + vloc;
  const int W = od.W, M1 = od.M1, M2 = od.M2, ld = od.ld1;
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + W * ld;
  C* tw = buf1 + W * ld;
  const C* tw1 = static_cast<const C*>(od.tw1);
  for (int i = threadIdx.x; i < M1; i += blockDim.x) tw[i] = tw1[i];
  for (int e = threadIdx.x; e < W * M1; e += blockDim.x) {
    const int c = e % W, j1 = e / W;
    const int j = M2 * j1 + cb * W + c;
    buf0[c * ld + j1] = load_a_pair(P, v, 2 * j, n, C{});
  }
  __syncthreads();
  C* res = fft_batch(buf0, buf1, M1, ld, W, od.rp1, tw);
  C* dst = static_cast<C*>(P.scratch) + od.scr_off + (int64_t)vloc * od.M;
  const C* tw4 = static_cast<const C*>(od.tw4);
  for (int e = threadIdx.x; e < W * M1; e += blockDim.x) {
    const int c = e % W, k1 = e / W, j2 = cb * W + c;
    dst[(int64_t)k1 * M2 + j2] = c_mul(res[c * ld + k1], tw4[j2 * k1]);
  }
}

// ---------------------------------------------------------------------------
// One block per row pair {k1a, M1 - k1a} of one order: both rows hold every
// spectrum index k together with its mirror M - k, which the real split needs.
template <class C>
__global__ void __launch_bounds__(kThreads) k_rows(const __grid_constant__ RhsParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int oi = find_order(P.rowpre, P.nord, blockIdx.x);
  const OrderDesc& od = P.ord[oi];
  const int kp = blockIdx.x - P.rowpre[oi];
  const int d = od.d, R = od.R, M1 = od.M1, M2 = od.M2, M = od.M, ld = od.ld2, G = od.G;
  const int k1a = kp, k1b = M1 - kp;
  const int nrow = (kp == 0 || 2 * kp == M1) ? 1 : 2;
  const int NP = nrow * M2;
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + G * 2 * ld;
  C* tw = buf1 + G * 2 * ld;
  const C* tw2 = static_cast<const C*>(od.tw2);
  const C* twL = static_cast<const C*>(od.twL);
  const C* src = static_cast<const C*>(P.scratch) + od.scr_off;
  for (int i = threadIdx.x; i < M2; i += blockDim.x) tw[i] = tw2[i];

  C S[kRowPosPerThread], Pr[kRowPosPerThread];
#pragma unroll
  for (int i = 0; i < kRowPosPerThread; ++i) {
    S[i] = c_zero(C{});
    Pr[i] = c_zero(C{});
  }
  C SN = c_zero(C{}), PrN = c_zero(C{});  // Nyquist index k = M (row 0 only)
  const bool nyq = (kp == 0 && threadIdx.x == 0);

  const int Vd = d * R;
  for (int q0 = 0; q0 < Vd; q0 += G) {
    const int gc = min(G, Vd - q0);
    for (int e = threadIdx.x; e < gc * NP; e += blockDim.x) {
      const int g = e / NP, p = e - g * NP;
      const int row = p / M2, pos = p - row * M2;
      const int q = q0 + g, r = q / d, m = q - r * d;
      const int k1 = row ? k1b : k1a;
      buf0[(g * nrow + row) * ld + pos] = src[(int64_t)(m * R + r) * M + (int64_t)k1 * M2 + pos];
    }
    __syncthreads();
    C* res = fft_batch(buf0, buf1, M2, ld, gc * nrow, od.rp2, tw);
#pragma unroll
    for (int i = 0; i < kRowPosPerThread; ++i) {
      const int p = threadIdx.x + i * blockDim.x;
      if (p < NP) {
        const int row = p / M2, pos = p - row * M2;
        const int k1 = row ? k1b : k1a;
        int mrow, mpos;
        if (k1 == 0) {
          mrow = row;
          mpos = pos == 0 ? 0 : M2 - pos;
        } else {
          mrow = (2 * k1 == M1) ? row : 1 - row;
          mpos = M2 - 1 - pos;
        }
        const C wL = twL[k1 + M1 * pos];
        for (int g = 0; g < gc; ++g) {
          const int q = q0 + g, r = q / d, m = q - r * d;
          const C A = unpack2(res[(g * nrow + row) * ld + pos], res[(g * nrow + mrow) * ld + mpos], wL);
          Pr[i] = (m == 0) ? A : c_mul(Pr[i], A);
          if (m == d - 1) S[i] = c_add(S[i], rank_weight(Pr[i], od, r));
        }
      }
    }
    if (nyq) {
      for (int g = 0; g < gc; ++g) {
        const int q = q0 + g, r = q / d, m = q - r * d;
        const C z0 = res[(g * nrow) * ld];
        const C zc = c_conj(z0);
        const C A = c_add(c_add(z0, zc), c_mul_pi(c_sub(z0, zc)));  // 2 A[M]
        PrN = (m == 0) ? A : c_mul(PrN, A);
        if (m == d - 1) SN = c_add(SN, rank_weight(PrN, od, r));
      }
    }
    __syncthreads();
  }

  // Inverse, row half: Z''[k] = (S[k] + S[k+M]) + i omega_L^-k (S[k] - S[k+M]),
  // S[k+M] = conj S[M-k] (Hermitian), S[M] for k = 0. The inverse transform is
  // run as a forward transform of conj(Z''); the final conjugation happens in
  // the column kernel.
  C* sS = buf1;  // NP + 1 entries
#pragma unroll
  for (int i = 0; i < kRowPosPerThread; ++i) {
    const int p = threadIdx.x + i * blockDim.x;
    if (p < NP) sS[p] = S[i];
  }
  if (nyq) sS[NP] = SN;
  __syncthreads();
  for (int p = threadIdx.x; p < NP; p += blockDim.x) {
    const int row = p / M2, pos = p - row * M2;
    const int k1 = row ? k1b : k1a;
    const int k = k1 + M1 * pos;
    int mp;
    if (k1 == 0) mp = row * M2 + (pos == 0 ? 0 : M2 - pos);
    else mp = ((2 * k1 == M1) ? row : 1 - row) * M2 + (M2 - 1 - pos);
    const C Sk = sS[p];
    const C Sm = (k == 0) ? sS[NP] : c_conj(sS[mp]);
    const C zpp = c_add(c_add(Sk, Sm), c_mul_pi(c_mul(c_conj(twL[k]), c_sub(Sk, Sm))));
    buf0[row * ld + pos] = c_conj(zpp);
  }
  __syncthreads();
  C* res = fft_batch(buf0, buf1, M2, ld, nrow, od.rp2, tw);
  C* dst = static_cast<C*>(P.scratch2) + od.scr2_off;
  const C* tw4 = static_cast<const C*>(od.tw4);
  for (int p = threadIdx.x; p < NP; p += blockDim.x) {
    const int row = p / M2, j2 = p - row * M2;
    const int k1 = row ? k1b : k1a;
    dst[(int64_t)k1 * M2 + j2] = c_mul(res[row * ld + j2], tw4[j2 * k1]);
  }
}

// ---------------------------------------------------------------------------
template <class C>
__global__ void __launch_bounds__(kThreads) k_inv_col(const __grid_constant__ RhsParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int oi = find_order(P.invpre, P.nord, blockIdx.x);
  const OrderDesc& od = P.ord[oi];
  const int cb = blockIdx.x - P.invpre[oi];
  const int W = od.W, M1 = od.M1, M2 = od.M2, ld = od.ld1, N = P.N;
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + W * ld;
  C* tw = buf1 + W * ld;
  const C* tw1 = static_cast<const C*>(od.tw1);
  for (int i = threadIdx.x; i < M1; i += blockDim.x) tw[i] = tw1[i];
  const C* src = static_cast<const C*>(P.scratch2) + od.scr2_off;
  for (int e = threadIdx.x; e < W * M1; e += blockDim.x) {
    const int c = e % W, k1 = e / W;
    buf0[c * ld + k1] = src[(int64_t)k1 * M2 + cb * W + c];
  }
  __syncthreads();
  C* res = fft_batch(buf0, buf1, M1, ld, W, od.rp1, tw);
  const double scale = ldexp(od.pscale, P.dwpath ? od.d * P.sc->e_n : 0);
  double* out = P.pd + (int64_t)oi * N;
  for (int e = threadIdx.x; e < W * M1; e += blockDim.x) {
    const int c = e % W, j1 = e / W;
    const int j = M2 * j1 + cb * W + c;
    const C w = res[c * ld + j1];
    const int k = 2 * j;  // sizes k (real part) and k + 1 (minus the imaginary part)
    if (k >= 1 && k <= N) out[k - 1] = cre(w) * scale;
    if (k + 1 <= N) out[k] = -cim(w) * scale;
  }
}

}  // namespace sag
