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

#include <type_traits>

#include "async_copy.cuh"
#include "dw_pow.cuh"
#include "fft_ct.cuh"
#include "plan.h"

namespace sag {

// ---- loading a = U o n, two sizes per complex point (k even) ---------------
// FP64: u, nn are the vector and the system's n, indexed by size - 1.
__device__ __forceinline__ cd load_a_pair(const double* __restrict__ u, const double* __restrict__ nn,
                                          int N, int k, cd) {
  double re = 0.0, im = 0.0;
  if (k >= 1 && k <= N) re = u[k - 1] * nn[k - 1];
  if (k + 1 <= N) im = u[k] * nn[k];
  return cd{re, im};
}
// Double-word: u, nn indexed by size, zero at size 0 and N + 1 and 16-byte
// aligned, so sizes k and k + 1 are one aligned 16-byte load of each.
__device__ __forceinline__ cdw load_a_pair(const float2* __restrict__ u, const float2* __restrict__ nn,
                                           int N, int k, cdw) {
  if (k > N) return c_zero(cdw{});
  const float4 a = __ldg(reinterpret_cast<const float4*>(u + k));
  const float4 b = __ldg(reinterpret_cast<const float4*>(nn + k));
  return make_cdw(dw_mul(dw{a.x, a.y}, dw{b.x, b.y}), dw_mul(dw{a.z, a.w}, dw{b.z, b.w}));
}
// Parametric factors (OrderDesc::pw): a = (u i^a) o n at sizes k and k + 1,
// the power generated in double-word (dw_pow.cuh) rather than loaded; up =
// the vector's (u 2^-e_v, a) as double-words.
__device__ __forceinline__ cdw gen_a_pair(const RhsParams& P, float4 up, const float2* __restrict__ nn, int N,
                                          int k) {
  if (k > N) return c_zero(cdw{});
  const float4 b = __ldg(reinterpret_cast<const float4*>(nn + k));
  const dw u{up.x, up.y}, a{up.z, up.w};
  const float2 l0 = __ldg(P.lnt + k);
  const dw re = dw_mul(dw_power(u, a, dw{l0.x, l0.y}, P.expk), dw{b.x, b.y});
  dw im{0.f, 0.f};
  if (k + 1 <= N) {
    const float2 l1 = __ldg(P.lnt + k + 1);
    im = dw_mul(dw_power(u, a, dw{l1.x, l1.y}, P.expk), dw{b.z, b.w});
  }
  return make_cdw(re, im);
}

__device__ __forceinline__ const double* vec_ptr(const RhsParams& P, int v, cd) { return P.U64 + P.voff[v]; }
__device__ __forceinline__ const float2* vec_ptr(const RhsParams& P, int v, cdw) {
  return P.Udw + P.vdwoff[v];
}
__device__ __forceinline__ const double* n_ptr(const RhsParams&, const double* n, const OrderDesc& od, cd) {
  return n + od.noff;
}
__device__ __forceinline__ const float2* n_ptr(const RhsParams& P, const double*, const OrderDesc& od, cdw) {
  return P.ndw + od.ndwoff;
}

// Power-of-two weight of a rank term (double-word path keeps every factor
// vector scaled to max |U| in [0.5, 1)); the FP64 path needs none.
__device__ __forceinline__ cd rank_weight(cd x, const OrderDesc&, int) { return x; }
__device__ __forceinline__ cdw rank_weight(cdw x, const OrderDesc& od, int r) {
  return c_scale2(x, od.rscale[r]);
}

// Spectrum slot of CP vector m R + r of an order (duplicates share one).
__device__ __forceinline__ int cp_slot(const RhsParams& P, const OrderDesc& od, int q) {
  return od.umap_off < 0 ? q : P.umap[od.umap_off + q];
}

// Twice the spectrum of a real sequence from its half-length packed transform:
// 2 A[k] = (Z[k] + conj Z[M-k]) - i omega_L^k (Z[k] - conj Z[M-k]).
template <class C>
__device__ __forceinline__ C unpack2(C zk, C zm, C wL) {
  C zc = c_conj(zm);
  return c_sub(c_add(zk, zc), c_mul_pi(c_mul(wL, c_sub(zk, zc))));
}

// Mirror of spectrum index k = k1 + M1 pos (row slot `row` of the block's
// row pair) at M - k, as (row slot, position).
__device__ __forceinline__ void mirror_of(int k1, int row, int pos, int M1, int M2, int& mrow,
                                          int& mpos) {
  if (k1 == 0) {
    mrow = row;
    mpos = pos == 0 ? 0 : M2 - pos;
  } else {
    mrow = (2 * k1 == M1) ? row : 1 - row;
    mpos = M2 - 1 - pos;
  }
}

// Epilogue of the compile-time column kernels: element e = c + W k1 of the
// block's W columns times its four-step twiddle tw4c[e], stored at row k1,
// column cb W + c of a row length `rowlen`. Each thread's W P1 / kThreads
// twiddles are loaded together first (the FFT's registers are free by now),
// so their L2 latency is paid once.
template <class C, int P1>
__device__ __forceinline__ void col_store_ct(const C* res, int ld, const C* __restrict__ tw4c, C* dst,
                                             int rowlen, int cb) {
  constexpr int W = ct_cols(P1), PE = W * P1 / kThreads;
  static_assert((W * P1) % kThreads == 0, "a column block is a whole number of thread sweeps");
  C w4[PE];
#pragma unroll
  for (int i = 0; i < PE; ++i) w4[i] = ld_ro(tw4c + threadIdx.x + i * kThreads);
#pragma unroll
  for (int i = 0; i < PE; ++i) {
    const int e = threadIdx.x + i * kThreads;
    const int c = e % W, k1 = e / W;
    dst[(int64_t)k1 * rowlen + cb * W + c] = c_mul(res[c * ld + pad8(k1)], w4[i]);
  }
}

// ---------------------------------------------------------------------------
// Forward column pass of one block: the order's vector lv (local index) into
// spectrum slot `slot`, column block cb. P1 > 0: compile-time length, in
// place; P1 == 0: runtime length, ping-pong.
template <class C, int P1, bool GEN = false>
__device__ __forceinline__ void fwd_col_body(const RhsParams& P, const OrderDesc& od, int slot, int lv,
                                             int cb, const double* __restrict__ n, C* buf) {
  constexpr bool CT = P1 > 0;
  const int M1 = CT ? P1 : od.M1;
  const int W = CT ? ct_cols(P1) : od.W;
  const int ld = CT ? ct_ld(P1, ct_cols(P1)) : od.ld1;
  const int M2 = od.M2;
  const int v = od.vbase + lv;
  C* buf1 = buf + W * ld;
  C* tw = buf1 + W * ld;  // runtime length only: the natural table in shared memory
  const C* tw1 = static_cast<const C*>(od.tw1);
  if constexpr (!CT)
    for (int i = threadIdx.x; i < M1; i += kThreads) tw[i] = tw1[i];
  const auto u = vec_ptr(P, v, C{});
  const auto nn = n_ptr(P, n, od, C{});
  const int N = od.N;
  float4 up{};
  if constexpr (GEN) up = __ldg(P.vpow + v);
  for (int e = threadIdx.x; e < W * M1; e += kThreads) {
    const int c = e % W, j1 = e / W;
    const int j = M2 * j1 + cb * W + c;
    C x;
    if constexpr (GEN) {
      x = gen_a_pair(P, up, nn, N, 2 * j);
    } else {
      x = load_a_pair(u, nn, N, 2 * j, C{});
    }
    buf[c * ld + (CT ? pad8(j1) : j1)] = x;
  }
  __syncthreads();
  C* res;
  if constexpr (CT) {
    // pass tables from global memory (no per-block fill)
    fft_ct<C, P1, ct_cols(P1), kThreads, true>(buf, ld, static_cast<const C*>(od.twg1));
    res = buf;
  } else {
    res = fft_batch(buf, buf1, M1, ld, W, od.rp1, tw);
  }
  C* dst = static_cast<C*>(P.scratch) + od.scr_off + (int64_t)slot * od.M;
  if constexpr (CT) {
    // four-step twiddles of this column block, stored in the loop's order
    col_store_ct<C, P1>(res, ld, static_cast<const C*>(od.tw4c) + (int64_t)cb * W * M1, dst, M2, cb);
  } else {
    const C* tw4 = static_cast<const C*>(od.tw4);
    for (int e = threadIdx.x; e < W * M1; e += kThreads) {
      const int c = e % W, k1 = e / W, j2 = cb * W + c;
      dst[(int64_t)k1 * M2 + j2] = c_mul(res[c * ld + k1], tw4[j2 * k1]);
    }
  }
}

// all = 0: each order's distinct vectors (colpre; duplicates share a slot);
// all = 1: every vector into its own slot (colpre_all; the adjoint).
// Forward column pass of a pair (double-word, compile-time length): vectors
// q = 2 pr, 2 pr + 1 of the order (rank-major, vector m R + r for q = r d + m)
// as the real and imaginary parts of one sequence indexed by size, j = 2 M2 j1
// + j2, so each complex point holds one size of each vector; column block cb
// of the M1 x 2 M2 geometry. A missing second vector (odd count) is zero.
template <class C, int P1, bool GEN = false>
__device__ __forceinline__ void fwd_col_pair_body(const RhsParams& P, const OrderDesc& od, int pr, int cb,
                                                  C* buf) {
  constexpr int W = ct_cols(P1);
  constexpr int ld = ct_ld(P1, W);
  constexpr ct_sched sc = make_ct_sched(P1);
  const int M2p = 2 * od.M2, N = od.N, d = od.d, R = od.R;
  const C* tw = static_cast<const C*>(od.twg1);  // pass tables, global layout
  const int q1 = 2 * pr, q2 = q1 + 1;
  const float2* nn = P.ndw + od.ndwoff;  // indexed by size, zero at 0
  // Pass 0 straight from the factors and n: point j1 of column c is size
  // j = 2 M2 j1 + cb W + c, z = (u1 n, u2 n) there (zero beyond N).
  if constexpr (GEN) {  // parametric factors: u i^a generated, ln j from the table
    const int v1 = od.vbase + (q1 % d) * R + q1 / d;
    const int v2 = q2 < od.nvec ? od.vbase + (q2 % d) * R + q2 / d : -1;
    const float4 up1 = __ldg(P.vpow + v1);
    const float4 up2 = v2 >= 0 ? __ldg(P.vpow + v2) : make_float4(0.f, 0.f, 0.f, 0.f);
    ct_pass_first_from<C, P1, W, kThreads>(
        [&](int c, int j1) -> C {
          const int j = M2p * j1 + cb * W + c;
          if (j > N) return c_zero(C{});
          const float2 nb = __ldg(nn + j), lj = __ldg(P.lnt + j);
          const dw nv{nb.x, nb.y}, l{lj.x, lj.y};
          dw im{0.f, 0.f};
          if (v2 >= 0) im = dw_mul(dw_power(dw{up2.x, up2.y}, dw{up2.z, up2.w}, l, P.expk), nv);
          return make_cdw(dw_mul(dw_power(dw{up1.x, up1.y}, dw{up1.z, up1.w}, l, P.expk), nv), im);
        },
        buf, ld);
  } else {
    const float2* u1 = P.Udw + P.vdwoff[od.vbase + (q1 % d) * R + q1 / d];
    const float2* u2 = q2 < od.nvec ? P.Udw + P.vdwoff[od.vbase + (q2 % d) * R + q2 / d] : nullptr;
    ct_pass_first_from<C, P1, W, kThreads>(
        [&](int c, int j1) -> C {
          const int j = M2p * j1 + cb * W + c;
          if (j > N) return c_zero(C{});
          const float2 nb = __ldg(nn + j), a1 = __ldg(u1 + j);
          const dw nv{nb.x, nb.y};
          dw im{0.f, 0.f};
          if (u2) {
            const float2 a2 = __ldg(u2 + j);
            im = dw_mul(dw{a2.x, a2.y}, nv);
          }
          return make_cdw(dw_mul(dw{a1.x, a1.y}, nv), im);
        },
        buf, ld);
  }
  ct_passes<C, P1, W, kThreads, 1, sc.r[0], true, sc.n - 1>(buf, ld, tw);  // middle passes, in place
  // The last pass hands each output k1 of column c, times its four-step
  // twiddle, straight to the workspace (row k1, column cb W + c of the
  // M1 x 2 M2 geometry).
  C* dst = static_cast<C*>(P.scratch) + od.scr_off + (int64_t)pr * 2 * od.M;
  const C* tw4c = static_cast<const C*>(od.tw4c_p) + (int64_t)cb * W * P1;
  ct_pass_last_to<C, P1, W, kThreads, true>(buf, ld, tw, [&](int c, int k1, C v) {
    dst[(int64_t)k1 * M2p + cb * W + c] = c_mul(v, ld_ro(tw4c + c + W * k1));
  });
}

// GEN: the double-word path's parametric factors (OrderDesc::pw), generated
// instead of read; a separate instantiation, so the stored-factor kernels keep
// their own register allocation.
template <class C, int KIND = kKindGeneral, bool GEN = false>
__global__ void __launch_bounds__(kThreads, 4) k_fwd_col(const __grid_constant__ RhsParams P,
                                                      const double* __restrict__ n, int base, int all) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int* pre = all ? P.colpre_all : P.colpre;
  const int bid = base + blockIdx.x;  // launches may cover a range of the table
  const int pos = find_segment(pre, P.nitems, bid);
  const int it = all ? pos : P.colperm[pos];  // colpre runs in colperm order
  const OrderDesc& od = P.ord[it];
  const int local = bid - pre[pos];
  if constexpr (KIND >= kKindPair) {  // every block of the launch: a pair at this column length
    const int pr = local / od.ncolblk_p, cbp = local - pr * od.ncolblk_p;
    fwd_col_pair_body<C, ct_len(KIND - kKindPair), GEN>(P, od, pr, cbp, buf);
    return;
  } else if constexpr (KIND != kKindGeneral) {  // single vectors, one length form
    const int vloc = local / od.ncolblk, cb = local - vloc * od.ncolblk;
    const int lv = (all || od.umap_off < 0) ? vloc : P.ulist[od.umap_off + vloc];
    fwd_col_body<C, KIND == kKindRuntime ? 0 : ct_len(KIND - kKindCt), GEN>(P, od, vloc, lv, cb, n, buf);
    return;
  }
  if constexpr (is_dw<C>::value) {
    if (!all && od.pair) {
      const int pr = local / od.ncolblk_p, cbp = local - pr * od.ncolblk_p;
      switch (od.M1) {
        case 64: fwd_col_pair_body<C, 64, GEN>(P, od, pr, cbp, buf); break;
        case 96: fwd_col_pair_body<C, 96, GEN>(P, od, pr, cbp, buf); break;
        case 128: fwd_col_pair_body<C, 128, GEN>(P, od, pr, cbp, buf); break;
        case 192: fwd_col_pair_body<C, 192, GEN>(P, od, pr, cbp, buf); break;
        case 256: fwd_col_pair_body<C, 256, GEN>(P, od, pr, cbp, buf); break;
        case 384: fwd_col_pair_body<C, 384, GEN>(P, od, pr, cbp, buf); break;
        case 512: fwd_col_pair_body<C, 512, GEN>(P, od, pr, cbp, buf); break;
        case 768: fwd_col_pair_body<C, 768, GEN>(P, od, pr, cbp, buf); break;
        case 1024: fwd_col_pair_body<C, 1024, GEN>(P, od, pr, cbp, buf); break;
        default: break;  // the plan sets pair only with a compile-time column length
      }
      return;
    }
  }
  const int vloc = local / od.ncolblk, cb = local - vloc * od.ncolblk;
  const int lv = (all || od.umap_off < 0) ? vloc : P.ulist[od.umap_off + vloc];
  if constexpr (!is_dw<C>::value) {
    fwd_col_body<C, 0, GEN>(P, od, vloc, lv, cb, n, buf);
    return;
  }
  switch (od.ct1 ? od.M1 : 0) {
    case 64: fwd_col_body<C, 64, GEN>(P, od, vloc, lv, cb, n, buf); break;
    case 96: fwd_col_body<C, 96, GEN>(P, od, vloc, lv, cb, n, buf); break;
    case 128: fwd_col_body<C, 128, GEN>(P, od, vloc, lv, cb, n, buf); break;
    case 192: fwd_col_body<C, 192, GEN>(P, od, vloc, lv, cb, n, buf); break;
    case 256: fwd_col_body<C, 256, GEN>(P, od, vloc, lv, cb, n, buf); break;
    case 384: fwd_col_body<C, 384, GEN>(P, od, vloc, lv, cb, n, buf); break;
    case 512: fwd_col_body<C, 512, GEN>(P, od, vloc, lv, cb, n, buf); break;
    case 768: fwd_col_body<C, 768, GEN>(P, od, vloc, lv, cb, n, buf); break;
    case 1024: fwd_col_body<C, 1024, GEN>(P, od, vloc, lv, cb, n, buf); break;
    case 1536: fwd_col_body<C, 1536, GEN>(P, od, vloc, lv, cb, n, buf); break;
    default: fwd_col_body<C, 0, GEN>(P, od, vloc, lv, cb, n, buf); break;
  }
}

// ---------------------------------------------------------------------------
// Row pass of one block: the row pair {k1a, M1 - k1a} of order od. Both rows
// hold every spectrum index k together with its mirror M - k, which the real
// split needs. Runtime row length (generic passes, ping-pong buffers).
template <class C>
__device__ __forceinline__ void rows_body(const RhsParams& P, const OrderDesc& od, int kp, C* buf) {
  // Positions per thread: the double-word path reaches this variant only for
  // rows of at most 128 points (the plan checks this), FP64 for up to 512.
  constexpr int PPT = is_dw<C>::value ? 1 : kRowPosPerThread;
  const int d = od.d, R = od.R, M1 = od.M1, M = od.M;
  const int M2 = od.M2;
  const int ld = od.ld2;
  const int G = od.G;
  const int k1a = kp, k1b = M1 - kp;
  const int nrow = (kp == 0 || 2 * kp == M1) ? 1 : 2;
  const int NP = nrow * M2;
  // Slots: transform (g, row) at buf + (g nrow + row) ld.
  C* buf1 = buf + G * 2 * ld;
  C* tw = buf1 + G * 2 * ld;
  const C* tw2 = static_cast<const C*>(od.tw2);
  const C* twL = static_cast<const C*>(od.twL);
  const C* src = static_cast<const C*>(P.scratch) + od.scr_off;
  for (int i = threadIdx.x; i < M2; i += kThreads) tw[i] = tw2[i];

  C S[PPT], Pr[PPT];
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    S[i] = c_zero(C{});
    Pr[i] = c_zero(C{});
  }
  C SN = c_zero(C{}), PrN = c_zero(C{});  // Nyquist index k = M (row 0 only)
  const bool nyq = (kp == 0 && threadIdx.x == 0);
  const int slot_stride = nrow;

  const int Vd = d * R;
  for (int q0 = 0; q0 < Vd; q0 += G) {
    const int gc = min(G, Vd - q0);
    for (int e = threadIdx.x; e < gc * NP; e += kThreads) {
      const int g = e / NP, p = e - g * NP;
      const int row = p / M2, pos = p - row * M2;
      const int q = q0 + g, r = q / d, m = q - r * d;
      const int k1 = row ? k1b : k1a;
      buf[(g * slot_stride + row) * ld + pos] = src[(int64_t)cp_slot(P, od, m * R + r) * M + (int64_t)k1 * M2 + pos];
    }
    __syncthreads();
    C* res = fft_batch(buf, buf1, M2, ld, gc * nrow, od.rp2, tw);
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const int p = threadIdx.x + i * kThreads;
      if (p < NP) {
        const int row = p / M2, pos = p - row * M2;
        const int k1 = row ? k1b : k1a;
        int mrow, mpos;
        mirror_of(k1, row, pos, M1, M2, mrow, mpos);
        const C wL = twL[k1 + M1 * pos];
        for (int g = 0; g < gc; ++g) {
          const int q = q0 + g, r = q / d, m = q - r * d;
          const C A = unpack2(res[(g * slot_stride + row) * ld + pos],
                              res[(g * slot_stride + mrow) * ld + mpos], wL);
          Pr[i] = (m == 0) ? A : C(c_mul(Pr[i], A));
          if (m == d - 1) S[i] = c_add(S[i], rank_weight(Pr[i], od, r));
        }
      }
    }
    if (nyq) {
      for (int g = 0; g < gc; ++g) {
        const int q = q0 + g, r = q / d, m = q - r * d;
        const C z0 = res[(g * slot_stride) * ld];
        const C zc = c_conj(z0);
        const C A = c_add(c_add(z0, zc), c_mul_pi(c_sub(z0, zc)));  // 2 A[M]
        PrN = (m == 0) ? A : C(c_mul(PrN, A));
        if (m == d - 1) SN = c_add(SN, rank_weight(PrN, od, r));
      }
    }
    __syncthreads();
  }

  // Inverse, row half: Z''[k] = (S[k] + S[k+M]) + i omega_L^-k (S[k] - S[k+M]),
  // S[k+M] = conj S[M-k] (Hermitian), S[M] for k = 0. The inverse transform is
  // run as a forward transform of conj(Z''); the final conjugation happens in
  // the column kernel. S is staged past the first two slots.
  C* sS = buf + 2 * ld;  // NP + 1 <= 2 ld entries, disjoint from slots 0 and 1
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int p = threadIdx.x + i * kThreads;
    if (p < NP) sS[p] = S[i];
  }
  if (nyq) sS[NP] = SN;
  __syncthreads();
  for (int p = threadIdx.x; p < NP; p += kThreads) {
    const int row = p / M2, pos = p - row * M2;
    const int k1 = row ? k1b : k1a;
    const int k = k1 + M1 * pos;
    int mrow, mpos;
    mirror_of(k1, row, pos, M1, M2, mrow, mpos);
    const C Sk = sS[p];
    const C Sm = (k == 0) ? sS[NP] : c_conj(sS[mrow * M2 + mpos]);
    const C zpp = c_add(c_add(Sk, Sm), c_mul_pi(c_mul(c_conj(twL[k]), c_sub(Sk, Sm))));
    buf[row * ld + pos] = c_conj(zpp);
  }
  __syncthreads();
  C* res = fft_batch(buf, buf1, M2, ld, nrow, od.rp2, tw);
  C* dst = static_cast<C*>(P.scratch2) + od.scr2_off;
  const C* tw4 = static_cast<const C*>(od.tw4);
  for (int p = threadIdx.x; p < NP; p += kThreads) {
    const int row = p / M2, j2 = p - row * M2;
    const int k1 = row ? k1b : k1a;
    dst[(int64_t)k1 * M2 + j2] = c_mul(res[row * ld + j2], tw4[j2 * k1]);
  }
}

// Row pass, compile-time row length. The rows of each chunk of G vectors
// (2 G transforms: both rows of the pair per vector) arrive by bulk
// asynchronous copies in natural order in a staging area; the first radix
// pass reads them from there and writes the padded work area, after which the
// block issues the copies of the next chunk, so they land while the remaining
// passes and the spectrum products of this chunk run. Layout: one mbarrier
// (16 bytes), stage (2 G x P2), work (2 G transforms, ct_ld(P2, 2 G) apart);
// the pass twiddle tables are read from global memory. If a copy does not
// complete within P.spin_limit cycles the block sets the timeout status, waits
// (bounded by kDrainLimit) for the copies it has in flight, and returns. The
// header's second 8 bytes hold a barrier nothing arrives at, which the waits
// target instead when P.wait_unmet is set (a test of that path).
template <class C, int P2>
__device__ __forceinline__ void rows_body_async(const RhsParams& P, const OrderDesc& od, int kp,
                                                unsigned char* smem_raw) {
  constexpr int G = ct_group(P2);
  constexpr int SLOTS = 2 * G;
  constexpr int ld = ct_ld(P2, SLOTS);
  constexpr int PPT = (2 * P2 + kThreads - 1) / kThreads;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  C* stage = reinterpret_cast<C*>(smem_raw + 16);
  C* work = stage + SLOTS * P2;
  const C* tw = static_cast<const C*>(od.twg2);  // pass tables, global memory
  const int d = od.d, R = od.R, M1 = od.M1, M = od.M;
  const int k1a = kp, k1b = M1 - kp;
  const int nrow = (kp == 0 || 2 * kp == M1) ? 1 : 2;
  const int NP = nrow * P2;
  const C* twL = static_cast<const C*>(od.twL);
  const C* src = static_cast<const C*>(P.scratch) + od.scr_off;
  const int Vd = d * R;
  const int nchunk = (Vd + G - 1) / G;

  // One thread issues the copies of chunk c: transform (g, row) at stage + (2 g + row) P2.
  auto issue = [&](int c) {
    const int q0 = c * G, gc = min(G, Vd - q0);
    mbar_arrive_expect_tx(bar, (uint32_t)(gc * nrow * P2 * sizeof(C)));
    for (int g = 0; g < gc; ++g) {
      const int q = q0 + g, r = q / d, m = q - r * d;
      for (int row = 0; row < nrow; ++row) {
        const int k1 = row ? k1b : k1a;
        bulk_copy_g2s(stage + (2 * g + row) * P2, src + (int64_t)cp_slot(P, od, m * R + r) * M + (int64_t)k1 * P2,
                      (uint32_t)(P2 * sizeof(C)), bar);
      }
    }
  };

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);  // the barrier nothing arrives at (P.wait_unmet)
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) issue(0);

  C S[PPT], Pr[PPT];
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    S[i] = c_zero(C{});
    Pr[i] = c_zero(C{});
  }
  C SN = c_zero(C{}), PrN = c_zero(C{});
  const bool nyq = (kp == 0 && threadIdx.x == 0);

  for (int c = 0; c < nchunk; ++c) {
    const int q0 = c * G, gc = min(G, Vd - q0);
    // The barrier also orders the previous chunk's reads of work before the
    // first pass overwrites it.
    // (a test of the timeout path waits on the barrier nothing completes)
    const bool ok = mbar_wait_bounded(P.wait_unmet ? bar + 1 : bar, (uint32_t)(c & 1), P.spin_limit);
    if (__syncthreads_or(!ok)) {
      // Timed out: latch the status, then let this chunk's copies land (a
      // second bounded wait) before the block's shared memory is released.
      if (threadIdx.x == 0) timeout_drain(P.status, kStatusTimeout, kStatusTimeoutUndrained, bar, (uint32_t)(c & 1));
      return;
    }
    fft_ct_first<C, P2, SLOTS, kThreads, true>(stage, P2, work, ld, tw);  // unused slots hold stale data
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0 && c + 1 < nchunk) issue(c + 1);
    fft_ct_rest<C, P2, SLOTS, kThreads, true>(work, ld, tw);
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const int p = threadIdx.x + i * kThreads;
      if (p < NP) {
        const int row = p / P2, pos = p - row * P2;
        const int k1 = row ? k1b : k1a;
        int mrow, mpos;
        mirror_of(k1, row, pos, M1, P2, mrow, mpos);
        const C wL = twL[k1 + M1 * pos];
        const int oa = row * ld + pad8(pos), ob = mrow * ld + pad8(mpos);
        for (int g = 0; g < gc; ++g) {
          const int q = q0 + g, r = q / d, m = q - r * d;
          const C* bg = work + 2 * g * ld;
          const C A = unpack2(bg[oa], bg[ob], wL);
          Pr[i] = (m == 0) ? A : C(c_mul(Pr[i], A));
          if (m == d - 1) S[i] = c_add(S[i], rank_weight(Pr[i], od, r));
        }
      }
    }
    if (nyq) {
      for (int g = 0; g < gc; ++g) {
        const int q = q0 + g, r = q / d, m = q - r * d;
        const C z0 = work[(2 * g) * ld];
        const C zc = c_conj(z0);
        const C A = c_add(c_add(z0, zc), c_mul_pi(c_sub(z0, zc)));  // 2 A[M]
        PrN = (m == 0) ? A : C(c_mul(PrN, A));
        if (m == d - 1) SN = c_add(SN, rank_weight(PrN, od, r));
      }
    }
  }

  // Inverse, row half (as in rows_body): S staged in the (idle) stage area,
  // the packed sequence built in work.
  C* sS = stage;
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int p = threadIdx.x + i * kThreads;
    if (p < NP) sS[p] = S[i];
  }
  if (nyq) sS[NP] = SN;
  __syncthreads();
  for (int p = threadIdx.x; p < NP; p += kThreads) {
    const int row = p / P2, pos = p - row * P2;
    const int k1 = row ? k1b : k1a;
    const int k = k1 + M1 * pos;
    int mrow, mpos;
    mirror_of(k1, row, pos, M1, P2, mrow, mpos);
    const C Sk = sS[p];
    const C Sm = (k == 0) ? sS[NP] : c_conj(sS[mrow * P2 + mpos]);
    const C zpp = c_add(c_add(Sk, Sm), c_mul_pi(c_mul(c_conj(twL[k]), c_sub(Sk, Sm))));
    work[row * ld + pad8(pos)] = c_conj(zpp);
  }
  __syncthreads();
  fft_ct<C, P2, 2, kThreads, true>(work, ld, tw);
  C* dst = static_cast<C*>(P.scratch2) + od.scr2_off;
  const C* tw4 = static_cast<const C*>(od.tw4);
  for (int p = threadIdx.x; p < NP; p += kThreads) {
    const int row = p / P2, j2 = p - row * P2;
    const int k1 = row ? k1b : k1a;
    dst[(int64_t)k1 * P2 + j2] = c_mul(work[row * ld + pad8(j2)], tw4[j2 * k1]);
  }
}

// Row pass of a CP order whose vectors repeat (a slot map, OrderDesc::
// umap_off >= 0; compile-time P2 = M2 points): block kp transforms the rows
// {k1a, M1 - k1a} of each distinct spectrum slot once, writing the real
// spectra 2 A[k] back in place and the Nyquist values to spec_nyq (as the TT
// row pass does); then it forms S = sum_r w_r prod_m A_{slot(m R + r)} at its
// points from those rows (its own writes, read back after the barrier), and
// ends with the inverse row half. The rank terms' d R uses of the spectra cost
// loads instead of row transforms. Layout: 16 bytes unused (the mbarrier slot
// of rows_body_async), then 2 G padded transforms; the inverse reuses them as
// the staged sums (2 P2 + 1) and two padded rows.
template <class C, int P2>
__device__ __forceinline__ void rows_body_dup(const RhsParams& P, const OrderDesc& od, int kp,
                                              unsigned char* smem_raw) {
  constexpr int G = ct_group(P2), SLOTS = 2 * G, ld = ct_ld(P2, SLOTS);
  constexpr int PPT = (2 * P2 + kThreads - 1) / kThreads;
  static_assert(2 * P2 + 1 <= (SLOTS - 2) * ld, "staged sums fit before the inverse rows");
  C* buf = reinterpret_cast<C*>(smem_raw + 16);
  const C* tw = static_cast<const C*>(od.twg2);
  const int d = od.d, R = od.R, M1 = od.M1, M = od.M;
  const int k1a = kp, k1b = M1 - kp;
  const int nrow = (kp == 0 || 2 * kp == M1) ? 1 : 2;
  const int NP = nrow * P2;
  const C* twL = static_cast<const C*>(od.twL);
  C* spec = static_cast<C*>(P.scratch) + od.scr_off;
  C* nyq = static_cast<C*>(P.spec_nyq) + od.vbase;
  for (int q0 = 0; q0 < od.nu; q0 += G) {
    const int gc = min(G, od.nu - q0);
    for (int e = threadIdx.x; e < gc * NP; e += kThreads) {
      const int g = e / NP, p = e - g * NP, row = p / P2, pos = p - row * P2;
      buf[(2 * g + row) * ld + pad8(pos)] = spec[(int64_t)(q0 + g) * M + (int64_t)(row ? k1b : k1a) * P2 + pos];
    }
    __syncthreads();
    fft_ct<C, P2, SLOTS, kThreads, true>(buf, ld, tw);  // slots without data hold stale values, unused
    for (int e = threadIdx.x; e < gc * NP; e += kThreads) {
      const int g = e / NP, p = e - g * NP, row = p / P2, pos = p - row * P2;
      const int k1 = row ? k1b : k1a;
      int mrow, mpos;
      mirror_of(k1, row, pos, M1, P2, mrow, mpos);
      const C* bg = buf + 2 * g * ld;
      spec[(int64_t)(q0 + g) * M + (int64_t)k1 * P2 + pos] =
          unpack2(bg[row * ld + pad8(pos)], bg[mrow * ld + pad8(mpos)], twL[k1 + M1 * pos]);
      if (k1 == 0 && pos == 0) {
        const C z0 = bg[0];
        const C zc = c_conj(z0);
        nyq[q0 + g] = c_add(c_add(z0, zc), c_mul_pi(c_sub(z0, zc)));  // 2 A[M]
      }
    }
    __syncthreads();
  }
  // Products and rank sum at the block's points, then staged for the inverse.
  C* sS = buf;
  C* work = buf + (SLOTS - 2) * ld;
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int p = threadIdx.x + i * kThreads;
    if (p < NP) {
      const int row = p / P2, pos = p - row * P2;
      const int64_t at = (int64_t)(row ? k1b : k1a) * P2 + pos;
      C S = c_zero(C{});
      for (int r = 0; r < R; ++r) {
        C Pr = spec[(int64_t)cp_slot(P, od, r) * M + at];
        for (int m = 1; m < d; ++m) Pr = c_mul(Pr, spec[(int64_t)cp_slot(P, od, m * R + r) * M + at]);
        S = c_add(S, rank_weight(Pr, od, r));
      }
      sS[p] = S;
    }
  }
  if (kp == 0 && threadIdx.x == 0) {
    C S = c_zero(C{});
    for (int r = 0; r < R; ++r) {
      C Pr = nyq[cp_slot(P, od, r)];
      for (int m = 1; m < d; ++m) Pr = c_mul(Pr, nyq[cp_slot(P, od, m * R + r)]);
      S = c_add(S, rank_weight(Pr, od, r));
    }
    sS[NP] = S;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < NP; p += kThreads) {
    const int row = p / P2, pos = p - row * P2;
    const int k1 = row ? k1b : k1a;
    const int k = k1 + M1 * pos;
    int mrow, mpos;
    mirror_of(k1, row, pos, M1, P2, mrow, mpos);
    const C Sk = sS[p];
    const C Sm = (k == 0) ? sS[NP] : c_conj(sS[mrow * P2 + mpos]);
    const C zpp = c_add(c_add(Sk, Sm), c_mul_pi(c_mul(c_conj(twL[k]), c_sub(Sk, Sm))));
    work[row * ld + pad8(pos)] = c_conj(zpp);
  }
  __syncthreads();
  fft_ct<C, P2, 2, kThreads, true>(work, ld, tw);
  C* dst = static_cast<C*>(P.scratch2) + od.scr2_off;
  const C* tw4 = static_cast<const C*>(od.tw4);
  for (int p = threadIdx.x; p < NP; p += kThreads) {
    const int row = p / P2, j2 = p - row * P2;
    const int k1 = row ? k1b : k1a;
    dst[(int64_t)k1 * P2 + j2] = c_mul(work[row * ld + pad8(j2)], tw4[j2 * k1]);
  }
}

// Row pass of the pair form (double-word, rows of P2p = 2 M2 points): block
// kp owns rows {k1, M1 - k1} of every pair's L-geometry transform, which hold
// every index k = k1 + M1 pos of row k1 together with its mirror L - k. The
// two vectors of a pair separate as 2 A1 = Z + conj Z(L-k) and
// 2 A2 = -i (Z - conj Z(L-k)); products and rank sums run over the P2p
// positions of row k1 only (row M1 - k1 is their Hermitian mirror). The
// inverse's row half then needs S(k) and S(k + M) of each M-geometry row,
// both in row k1 or, conjugated, in its mirror. Layout: one mbarrier (16
// bytes), stage (2 G x P2p), work (2 G transforms, ct_ld(P2p, 2 G) apart). The
// pass twiddles come from global tables (ct_twg layout), which keeps the block
// at three per SM for 512-point rows.
template <class C, int P2p>
__device__ __forceinline__ void rows_body_pair(const RhsParams& P, const OrderDesc& od, int kp,
                                               unsigned char* smem_raw) {
  constexpr int M2c = P2p / 2;
  constexpr int G = ct_group(P2p);  // pairs per chunk
  constexpr int SLOTS = 2 * G;
  constexpr int ld = ct_ld(P2p, SLOTS);
  constexpr int ldi = ct_ld(M2c, 2);
  static_assert(2 * ldi <= SLOTS * ld, "inverse rows fit the work area");
  constexpr int PPT = (P2p + kThreads - 1) / kThreads;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  C* stage = reinterpret_cast<C*>(smem_raw + 16);
  C* work = stage + SLOTS * P2p;
  const C* tw = static_cast<const C*>(od.tw2p);
  const C* twi = static_cast<const C*>(od.twg2);
  const int d = od.d, R = od.R, M1 = od.M1, M = od.M;
  const int k1a = kp, k1b = M1 - kp;
  const int nrow = (kp == 0 || 2 * kp == M1) ? 1 : 2;
  const C* twL = static_cast<const C*>(od.twL);
  const C* src = static_cast<const C*>(P.scratch) + od.scr_off;  // pair p at src + 2 M p
  const int Vd = d * R, np = od.npair;
  const int nchunk = (np + G - 1) / G;

  auto issue = [&](int c) {
    const int p0 = c * G, gc = min(G, np - p0);
    mbar_arrive_expect_tx(bar, (uint32_t)(gc * nrow * P2p * sizeof(C)));
    for (int g = 0; g < gc; ++g)
      for (int row = 0; row < nrow; ++row) {
        const int k1 = row ? k1b : k1a;
        bulk_copy_g2s(stage + (2 * g + row) * P2p, src + (int64_t)(p0 + g) * 2 * M + (int64_t)k1 * P2p,
                      (uint32_t)(P2p * sizeof(C)), bar);
      }
  };

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);  // the barrier nothing arrives at (P.wait_unmet)
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) issue(0);

  C S[PPT], Pr[PPT];
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    S[i] = c_zero(C{});
    Pr[i] = c_zero(C{});
  }
  auto accumulate = [&](int i, const C& A, int q) {
    const int r = q / d, m = q - r * d;
    Pr[i] = (m == 0) ? A : C(c_mul(Pr[i], A));
    if (m == d - 1) S[i] = c_add(S[i], rank_weight(Pr[i], od, r));
  };

  for (int c = 0; c < nchunk; ++c) {
    const int p0 = c * G, gc = min(G, np - p0);
    // (a test of the timeout path waits on the barrier nothing completes)
    const bool ok = mbar_wait_bounded(P.wait_unmet ? bar + 1 : bar, (uint32_t)(c & 1), P.spin_limit);
    if (__syncthreads_or(!ok)) {
      // Timed out: latch the status, then let this chunk's copies land (a
      // second bounded wait) before the block's shared memory is released.
      if (threadIdx.x == 0) timeout_drain(P.status, kStatusTimeout, kStatusTimeoutUndrained, bar, (uint32_t)(c & 1));
      return;
    }
    if (od.discard) {
      // The chunk's rows are in shared memory and no kernel reads them again
      // (each row belongs to one block): their L2 lines go without a write-back.
      constexpr int LPR = P2p * (int)sizeof(C) / 128;  // lines per row
      for (int e = threadIdx.x; e < gc * nrow * LPR; e += kThreads) {
        const int rr = e / LPR, ln = e - rr * LPR, g = rr / nrow, row = rr - g * nrow;
        discard_l2(src + (int64_t)(p0 + g) * 2 * M + (int64_t)(row ? k1b : k1a) * P2p + ln * (128 / (int)sizeof(C)));
      }
    }
    fft_ct_first<C, P2p, SLOTS, kThreads, true>(stage, P2p, work, ld, tw);  // unused slots hold stale data
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0 && c + 1 < nchunk) issue(c + 1);
    fft_ct_rest<C, P2p, SLOTS, kThreads, true>(work, ld, tw);
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const int p = threadIdx.x + i * kThreads;
      if (p < P2p) {
        int mrow, mpos;
        mirror_of(k1a, 0, p, M1, P2p, mrow, mpos);
        const int oa = pad8(p), ob = mrow * ld + pad8(mpos);
        for (int g = 0; g < gc; ++g) {
          const C* bg = work + 2 * g * ld;
          const C z = bg[oa], zc = c_conj(bg[ob]);
          const int q = 2 * (p0 + g);
          accumulate(i, c_add(z, zc), q);
          if (q + 1 < Vd) accumulate(i, c_mul_mi(c_sub(z, zc)), q + 1);
        }
      }
    }
    __syncthreads();
  }

  // Inverse, row half: S of row k1 staged in the (idle) stage area; the packed
  // sequences of M-geometry rows k1 (and M1 - k1) built in work.
  C* sS = stage;
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int p = threadIdx.x + i * kThreads;
    if (p < P2p) sS[p] = S[i];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nrow * M2c; e += kThreads) {
    const int row = e / M2c, k2 = e - row * M2c;
    const int k1 = row ? k1b : k1a;
    const int k = k1 + M1 * k2;
    C Sk, SkM;  // S(k), S(k + M)
    if (row == 0) {
      Sk = sS[k2];
      SkM = sS[k2 + M2c];
    } else {
      Sk = c_conj(sS[P2p - 1 - k2]);
      SkM = c_conj(sS[M2c - 1 - k2]);
    }
    const C zpp = c_add(c_add(Sk, SkM), c_mul_pi(c_mul(c_conj(twL[k]), c_sub(Sk, SkM))));
    work[row * ldi + pad8(k2)] = c_conj(zpp);
  }
  __syncthreads();
  fft_ct<C, M2c, 2, kThreads, true>(work, ldi, twi);
  C* dst = static_cast<C*>(P.scratch2) + od.scr2_off;
  const C* tw4 = static_cast<const C*>(od.tw4);
  for (int e = threadIdx.x; e < nrow * M2c; e += kThreads) {
    const int row = e / M2c, j2 = e - row * M2c;
    const int k1 = row ? k1b : k1a;
    dst[(int64_t)k1 * M2c + j2] = c_mul(work[row * ldi + pad8(j2)], tw4[j2 * k1]);
  }
}

template <class C, int KIND = kKindGeneral>
__global__ void __launch_bounds__(kThreads, 3) k_rows(const __grid_constant__ RhsParams P, int base) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  // Items with the most vectors per row pair come first (rowperm), so that
  // they are scheduled first; launches may cover a range of the table.
  const int bid = base + blockIdx.x;
  const int j = find_segment(P.rowpre, P.nitems, bid);
  const OrderDesc& od = P.ord[P.rowperm[j]];
  const int kp = bid - P.rowpre[j];
  if constexpr (KIND >= kKindPair) {
    rows_body_pair<C, ct_len(KIND - kKindPair)>(P, od, kp, smem_raw);
    return;
  } else if constexpr (KIND >= kKindCt) {
    if (od.umap_off >= 0) rows_body_dup<C, ct_len(KIND - kKindCt)>(P, od, kp, smem_raw);
    else rows_body_async<C, ct_len(KIND - kKindCt)>(P, od, kp, smem_raw);
    return;
  } else if constexpr (KIND == kKindRuntime) {
    rows_body<C>(P, od, kp, buf);
    return;
  }
  if constexpr (!is_dw<C>::value) {
    rows_body<C>(P, od, kp, buf);
    return;
  }
  if (od.pair) {
    switch (2 * od.M2) {
      case 128: rows_body_pair<C, 128>(P, od, kp, smem_raw); break;
      case 256: rows_body_pair<C, 256>(P, od, kp, smem_raw); break;
      case 512: rows_body_pair<C, 512>(P, od, kp, smem_raw); break;
      default: break;  // the plan sets pair only for these row lengths
    }
    return;
  }
  if (od.ct2 && od.umap_off >= 0) {
    switch (od.M2) {
      case 64: rows_body_dup<C, 64>(P, od, kp, smem_raw); return;
      case 128: rows_body_dup<C, 128>(P, od, kp, smem_raw); return;
      case 256: rows_body_dup<C, 256>(P, od, kp, smem_raw); return;
      case 512: rows_body_dup<C, 512>(P, od, kp, smem_raw); return;
      default: break;
    }
  }
  switch (od.ct2 ? od.M2 : 0) {
    case 64: rows_body_async<C, 64>(P, od, kp, smem_raw); break;
    case 128: rows_body_async<C, 128>(P, od, kp, smem_raw); break;
    case 256: rows_body_async<C, 256>(P, od, kp, smem_raw); break;
    case 512: rows_body_async<C, 512>(P, od, kp, smem_raw); break;
    default: rows_body<C>(P, od, kp, buf); break;
  }
}

// ---------------------------------------------------------------------------
// Inverse column pass: column block cb of order od; keeps sizes 1..N.
template <class C, int P1>
__device__ __forceinline__ void inv_col_body(const RhsParams& P, const OrderDesc& od, int oi, int cb,
                                             C* buf) {
  constexpr bool CT = P1 > 0;
  const int M1 = CT ? P1 : od.M1;
  const int W = CT ? ct_cols(P1) : od.W;
  const int ld = CT ? ct_ld(P1, ct_cols(P1)) : od.ld1;
  const int M2 = od.M2, N = od.N;
  C* buf1 = buf + W * ld;
  C* tw = buf1 + W * ld;  // runtime length only: the natural table in shared memory
  const C* tw1 = static_cast<const C*>(od.tw1);
  if constexpr (!CT)
    for (int i = threadIdx.x; i < M1; i += kThreads) tw[i] = tw1[i];
  const C* src = static_cast<const C*>(P.scratch2) + od.scr2_off;
  const double scale = ldexp(od.pscale, P.dwpath ? od.d * P.sc[od.sys].e_n : 0);
  double* out = P.pd + od.pd_off;
  if constexpr (CT) {
    // First pass straight from the spectrum rows, last pass straight to the
    // kept outputs (column c, point j1 is index j = M2 j1 + cb W + c: sizes
    // 2 j and 2 j + 1); pass tables from global memory.
    constexpr ct_sched sc = make_ct_sched(P1);
    const C* twg = static_cast<const C*>(od.twg1);
    ct_pass_first_from<C, P1, ct_cols(P1), kThreads>(
        [&](int c, int k1) -> C { return ld_ro(src + (int64_t)k1 * M2 + cb * W + c); }, buf, ld);
    ct_passes<C, P1, ct_cols(P1), kThreads, 1, sc.r[0], true, sc.n - 1>(buf, ld, twg);
    ct_pass_last_to<C, P1, ct_cols(P1), kThreads, true>(buf, ld, twg, [&](int c, int j1, C w) {
      const int k = 2 * (M2 * j1 + cb * W + c);
      if (k >= 1 && k <= N) out[k - 1] = cre(w) * scale;
      if (k + 1 <= N) out[k] = -cim(w) * scale;
    });
  } else {
    for (int e = threadIdx.x; e < W * M1; e += kThreads) {
      const int c = e % W, k1 = e / W;
      buf[c * ld + k1] = src[(int64_t)k1 * M2 + cb * W + c];
    }
    __syncthreads();
    C* res = fft_batch(buf, buf1, M1, ld, W, od.rp1, tw);
    for (int e = threadIdx.x; e < W * M1; e += kThreads) {
      const int c = e % W, j1 = e / W;
      const int j = M2 * j1 + cb * W + c;
      const C w = res[c * ld + j1];
      const int k = 2 * j;  // sizes k (real part) and k + 1 (minus the imaginary part)
      if (k >= 1 && k <= N) out[k - 1] = cre(w) * scale;
      if (k + 1 <= N) out[k] = -cim(w) * scale;
    }
  }
}

template <class C, int KIND = kKindGeneral>
__global__ void __launch_bounds__(kThreads, 4) k_inv_col(const __grid_constant__ RhsParams P, int base) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int bid = base + blockIdx.x;  // launches may cover a range of the invpre table
  const int oi = find_segment(P.invpre, P.nitems, bid);
  const OrderDesc& od = P.ord[oi];
  const int cb = bid - P.invpre[oi];
  if constexpr (KIND >= kKindCt) {
    inv_col_body<C, ct_len(KIND - kKindCt)>(P, od, oi, cb, buf);
    return;
  } else if constexpr (KIND == kKindRuntime) {
    inv_col_body<C, 0>(P, od, oi, cb, buf);
    return;
  }
  if constexpr (!is_dw<C>::value) {
    inv_col_body<C, 0>(P, od, oi, cb, buf);
    return;
  }
  switch (od.ct1 ? od.M1 : 0) {
    case 64: inv_col_body<C, 64>(P, od, oi, cb, buf); break;
    case 96: inv_col_body<C, 96>(P, od, oi, cb, buf); break;
    case 128: inv_col_body<C, 128>(P, od, oi, cb, buf); break;
    case 192: inv_col_body<C, 192>(P, od, oi, cb, buf); break;
    case 256: inv_col_body<C, 256>(P, od, oi, cb, buf); break;
    case 384: inv_col_body<C, 384>(P, od, oi, cb, buf); break;
    case 512: inv_col_body<C, 512>(P, od, oi, cb, buf); break;
    case 768: inv_col_body<C, 768>(P, od, oi, cb, buf); break;
    case 1024: inv_col_body<C, 1024>(P, od, oi, cb, buf); break;
    case 1536: inv_col_body<C, 1536>(P, od, oi, cb, buf); break;
    default: inv_col_body<C, 0>(P, od, oi, cb, buf); break;
  }
}

}  // namespace sag

// ===========================================================================
// TT kernels (Eq. ch3.eq4). The forward column pass is shared with CP; the
// spectra of the nonzero core vectors are then combined per frequency by the
// matrix chain S_d[k] = e_0 A^(1)[k] A^(2)[k] ... A^(d)[k] e_0, where
// A^(l)_{a,b}[k] is the spectrum of h^(l)_{a,b} o n (Sec. 3 stores the cores as
// these vectors along the size axis).
namespace sag {

// Row pass of the TT path: row FFTs of every vector of the order at the row
// pair {k1a, M1 - k1a}, split into real spectra 2 A[k] written back in place
// (same rows of the workspace); the Nyquist value goes to spec_nyq.
// The same pass with compile-time M2-point transforms (double-word, OrderDesc::
// ctt): chunks of ct_group(M2) vectors, their two rows in the padded layout
// (slot 2 g + row; a single-row block leaves the odd slots stale and unused),
// transformed in place with the pass tables in global memory.
template <class C, int P2>
__device__ __forceinline__ void rows_tt_fwd_ct(const RhsParams& P, const OrderDesc& od, int kp, C* buf) {
  constexpr int G = ct_group(P2), SLOTS = 2 * G, ld = ct_ld(P2, SLOTS);
  const C* tw = static_cast<const C*>(od.twg2);
  const int M1 = od.M1, M = od.M;
  const int k1a = kp, k1b = M1 - kp;
  const int nrow = (kp == 0 || 2 * kp == M1) ? 1 : 2;
  const int NP = nrow * P2;
  const C* twL = static_cast<const C*>(od.twL);
  C* spec = static_cast<C*>(P.scratch) + od.scr_off;
  C* nyq = static_cast<C*>(P.spec_nyq) + od.vbase;
  for (int q0 = 0; q0 < od.nvec; q0 += G) {
    const int gc = min(G, od.nvec - q0);
    for (int e = threadIdx.x; e < gc * NP; e += kThreads) {
      const int g = e / NP, p = e - g * NP, row = p / P2, pos = p - row * P2;
      buf[(2 * g + row) * ld + pad8(pos)] = spec[(int64_t)(q0 + g) * M + (int64_t)(row ? k1b : k1a) * P2 + pos];
    }
    __syncthreads();
    fft_ct<C, P2, SLOTS, kThreads, true>(buf, ld, tw);
    for (int e = threadIdx.x; e < gc * NP; e += kThreads) {
      const int g = e / NP, p = e - g * NP, row = p / P2, pos = p - row * P2;
      const int k1 = row ? k1b : k1a;
      int mrow, mpos;
      mirror_of(k1, row, pos, M1, P2, mrow, mpos);
      const C* bg = buf + 2 * g * ld;
      spec[(int64_t)(q0 + g) * M + (int64_t)k1 * P2 + pos] =
          unpack2(bg[row * ld + pad8(pos)], bg[mrow * ld + pad8(mpos)], twL[k1 + M1 * pos]);
      if (k1 == 0 && pos == 0) {
        const C z0 = bg[0];
        const C zc = c_conj(z0);
        nyq[q0 + g] = c_add(c_add(z0, zc), c_mul_pi(c_sub(z0, zc)));  // 2 A[M]
      }
    }
    __syncthreads();
  }
}

template <class C>
__global__ void __launch_bounds__(kThreads, 3) k_rows_tt_fwd(const __grid_constant__ RhsParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int j = find_segment(P.rowpre, P.nitems, blockIdx.x);
  const int oi = P.rowperm[j];
  const OrderDesc& od = P.ord[oi];
  const int kp = blockIdx.x - P.rowpre[j];
  if constexpr (is_dw<C>::value) {
    if (od.ctt) {
      switch (od.M2) {
        case 64: rows_tt_fwd_ct<C, 64>(P, od, kp, buf); return;
        case 128: rows_tt_fwd_ct<C, 128>(P, od, kp, buf); return;
        case 256: rows_tt_fwd_ct<C, 256>(P, od, kp, buf); return;
        case 512: rows_tt_fwd_ct<C, 512>(P, od, kp, buf); return;
        default: break;  // the plan sets ctt only for these lengths (M2 is a power of two)
      }
    }
  }
  const int M1 = od.M1, M2 = od.M2, M = od.M, ld = od.ld2, G = od.G;
  const int k1a = kp, k1b = M1 - kp;
  const int nrow = (kp == 0 || 2 * kp == M1) ? 1 : 2;
  const int NP = nrow * M2;
  C* buf1 = buf + G * 2 * ld;
  C* tw = buf1 + G * 2 * ld;
  const C* tw2 = static_cast<const C*>(od.tw2);
  const C* twL = static_cast<const C*>(od.twL);
  C* spec = static_cast<C*>(P.scratch) + od.scr_off;
  C* nyq = static_cast<C*>(P.spec_nyq) + od.vbase;
  for (int i = threadIdx.x; i < M2; i += kThreads) tw[i] = tw2[i];
  for (int q0 = 0; q0 < od.nvec; q0 += G) {
    const int gc = min(G, od.nvec - q0);
    for (int e = threadIdx.x; e < gc * NP; e += kThreads) {
      const int g = e / NP, p = e - g * NP;
      const int row = p / M2, pos = p - row * M2;
      const int k1 = row ? k1b : k1a;
      buf[(g * nrow + row) * ld + pos] = spec[(int64_t)(q0 + g) * M + (int64_t)k1 * M2 + pos];
    }
    __syncthreads();
    C* res = fft_batch(buf, buf1, M2, ld, gc * nrow, od.rp2, tw);
    for (int e = threadIdx.x; e < gc * NP; e += kThreads) {
      const int g = e / NP, p = e - g * NP;
      const int row = p / M2, pos = p - row * M2;
      const int k1 = row ? k1b : k1a;
      int mrow, mpos;
      mirror_of(k1, row, pos, M1, M2, mrow, mpos);
      const C A = unpack2(res[(g * nrow + row) * ld + pos], res[(g * nrow + mrow) * ld + mpos],
                          twL[k1 + M1 * pos]);
      spec[(int64_t)(q0 + g) * M + (int64_t)k1 * M2 + pos] = A;
      if (k1 == 0 && pos == 0) {
        const C z0 = res[(g * nrow + row) * ld];
        const C zc = c_conj(z0);
        nyq[q0 + g] = c_add(c_add(z0, zc), c_mul_pi(c_sub(z0, zc)));  // 2 A[M]
      }
    }
    __syncthreads();
  }
}

// Power-of-two weight of core entry j (index into the plan's vid table).
__device__ __forceinline__ cd tt_weight(cd x, const RhsParams&, int) { return x; }
__device__ __forceinline__ cdw tt_weight(cdw x, const RhsParams& P, int j) {
  return c_scale2(x, P.ewt[j]);
}

// Per-frequency matrix chain of one order; thread e < M handles the spectrum
// slot e (same [k1][k2] layout as the vectors' spectra), e = M the Nyquist.
template <class C, int RMAX>
__global__ void __launch_bounds__(256) k_tt_chain(const __grid_constant__ RhsParams P) {
  const int oi = find_segment(P.chainpre, P.nitems, blockIdx.x);
  const OrderDesc& od = P.ord[oi];
  const int e = (blockIdx.x - P.chainpre[oi]) * blockDim.x + threadIdx.x;
  const int M = od.M;
  if (e > M) return;
  const C* spec = static_cast<const C*>(P.scratch) + od.scr_off;
  const C* nyq = static_cast<const C*>(P.spec_nyq);
  const int* vid = P.vid + od.vid_off;
  auto load = [&](int j) -> C {  // core entry j of the order, its vector vid[j] >= 0
    const int v = vid[j];
    const C z = (e < M) ? spec[(int64_t)(v - od.vbase) * M + e] : nyq[v];
    return tt_weight(z, P, od.vid_off + j);
  };
  C x[RMAX], xn[RMAX];
  const int r1 = od.ttr[1];
#pragma unroll
  for (int b = 0; b < RMAX; ++b) {
    x[b] = c_zero(C{});
    if (b < r1 && vid[b] >= 0) x[b] = load(b);
  }
  int off = r1;
  for (int l = 2; l <= od.d; ++l) {
    const int ra = od.ttr[l - 1], rb = od.ttr[l];
#pragma unroll
    for (int b = 0; b < RMAX; ++b) {
      xn[b] = c_zero(C{});
      if (b < rb) {
#pragma unroll
        for (int a = 0; a < RMAX; ++a) {
          if (a < ra) {
            const int j = off + a * rb + b;
            if (vid[j] >= 0) xn[b] = c_add(xn[b], c_mul(x[a], load(j)));
          }
        }
      }
    }
#pragma unroll
    for (int b = 0; b < RMAX; ++b) x[b] = xn[b];
    off += ra * rb;
  }
  if (e < M) static_cast<C*>(P.scratch2)[od.scr2_off + e] = x[0];
  else static_cast<C*>(P.s_nyq)[oi] = x[0];
}

// Inverse row half of the TT path: repack the spectral sum of rows
// {k1a, M1 - k1a} (with its Nyquist value), inverse row FFTs, four-step
// twiddle, written back in place for the inverse column kernel.
// The same with compile-time transforms (OrderDesc::ctt): sums staged at buf,
// the two packed rows in the padded layout after them.
template <class C, int P2>
__device__ __forceinline__ void rows_tt_inv_ct(const RhsParams& P, const OrderDesc& od, int oi, int kp, C* buf) {
  constexpr int ldi = ct_ld(P2, 2);
  const int M1 = od.M1;
  const int k1a = kp, k1b = M1 - kp;
  const int nrow = (kp == 0 || 2 * kp == M1) ? 1 : 2;
  const int NP = nrow * P2;
  C* sS = buf;
  C* work = buf + 2 * P2;
  const C* twL = static_cast<const C*>(od.twL);
  C* S = static_cast<C*>(P.scratch2) + od.scr2_off;
  const C SM = static_cast<const C*>(P.s_nyq)[oi];
  for (int p = threadIdx.x; p < NP; p += kThreads) {
    const int row = p / P2, pos = p - row * P2;
    sS[p] = S[(int64_t)(row ? k1b : k1a) * P2 + pos];
  }
  __syncthreads();
  for (int p = threadIdx.x; p < NP; p += kThreads) {
    const int row = p / P2, pos = p - row * P2;
    const int k1 = row ? k1b : k1a;
    const int k = k1 + M1 * pos;
    int mrow, mpos;
    mirror_of(k1, row, pos, M1, P2, mrow, mpos);
    const C Sk = sS[p];
    const C Sm = (k == 0) ? SM : C(c_conj(sS[mrow * P2 + mpos]));
    const C zpp = c_add(c_add(Sk, Sm), c_mul_pi(c_mul(c_conj(twL[k]), c_sub(Sk, Sm))));
    work[row * ldi + pad8(pos)] = c_conj(zpp);
  }
  __syncthreads();
  fft_ct<C, P2, 2, kThreads, true>(work, ldi, static_cast<const C*>(od.twg2));
  const C* tw4 = static_cast<const C*>(od.tw4);
  for (int p = threadIdx.x; p < NP; p += kThreads) {
    const int row = p / P2, j2 = p - row * P2;
    const int k1 = row ? k1b : k1a;
    S[(int64_t)k1 * P2 + j2] = c_mul(work[row * ldi + pad8(j2)], tw4[j2 * k1]);
  }
}

template <class C>
__global__ void __launch_bounds__(kThreads, 3) k_rows_tt_inv(const __grid_constant__ RhsParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int j = find_segment(P.rowpre, P.nitems, blockIdx.x);
  const int oi = P.rowperm[j];
  const OrderDesc& od = P.ord[oi];
  const int kp = blockIdx.x - P.rowpre[j];
  if constexpr (is_dw<C>::value) {
    if (od.ctt) {
      switch (od.M2) {
        case 64: rows_tt_inv_ct<C, 64>(P, od, oi, kp, buf); return;
        case 128: rows_tt_inv_ct<C, 128>(P, od, oi, kp, buf); return;
        case 256: rows_tt_inv_ct<C, 256>(P, od, oi, kp, buf); return;
        case 512: rows_tt_inv_ct<C, 512>(P, od, oi, kp, buf); return;
        default: break;
      }
    }
  }
  const int M1 = od.M1, M2 = od.M2, ld = od.ld2;
  const int k1a = kp, k1b = M1 - kp;
  const int nrow = (kp == 0 || 2 * kp == M1) ? 1 : 2;
  const int NP = nrow * M2;
  C* sS = buf;               // NP staged spectral sums
  C* bufa = buf + 2 * ld;    // two transform slots
  C* bufb = bufa + 2 * ld;
  C* tw = bufb + 2 * ld;
  const C* tw2 = static_cast<const C*>(od.tw2);
  const C* twL = static_cast<const C*>(od.twL);
  C* S = static_cast<C*>(P.scratch2) + od.scr2_off;
  const C SM = static_cast<const C*>(P.s_nyq)[oi];
  for (int i = threadIdx.x; i < M2; i += kThreads) tw[i] = tw2[i];
  for (int p = threadIdx.x; p < NP; p += kThreads) {
    const int row = p / M2, pos = p - row * M2;
    sS[p] = S[(int64_t)(row ? k1b : k1a) * M2 + pos];
  }
  __syncthreads();
  for (int p = threadIdx.x; p < NP; p += kThreads) {
    const int row = p / M2, pos = p - row * M2;
    const int k1 = row ? k1b : k1a;
    const int k = k1 + M1 * pos;
    int mrow, mpos;
    mirror_of(k1, row, pos, M1, M2, mrow, mpos);
    const C Sk = sS[p];
    const C Sm = (k == 0) ? SM : C(c_conj(sS[mrow * M2 + mpos]));
    const C zpp = c_add(c_add(Sk, Sm), c_mul_pi(c_mul(c_conj(twL[k]), c_sub(Sk, Sm))));
    bufa[row * ld + pos] = c_conj(zpp);
  }
  __syncthreads();
  C* res = fft_batch(bufa, bufb, M2, ld, nrow, od.rp2, tw);
  const C* tw4 = static_cast<const C*>(od.tw4);
  for (int p = threadIdx.x; p < NP; p += kThreads) {
    const int row = p / M2, j2 = p - row * M2;
    const int k1 = row ? k1b : k1a;
    S[(int64_t)k1 * M2 + j2] = c_mul(res[row * ld + j2], tw4[j2 * k1]);
  }
}

}  // namespace sag
