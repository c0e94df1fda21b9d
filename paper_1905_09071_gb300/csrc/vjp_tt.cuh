// Vector-Jacobian product of the TT right-hand side (Eq. ch3.eq4), templated
// on the complex scalar.
//
// Gain: per frequency the order's spectral sum is the matrix chain
// S = A_1 A_2 ... A_d (1 x R_1, R_1 x R_2, ..., R_{d-1} x 1) of the cores'
// spectra A_l[a, b] = FFT(h^(l)_{a,b} o n). The cotangent of the sequence
// h^(l)_{a,b} o n is the correlation of g with the product of every other
// core, whose spectrum is G conj(pre_{l-1}[a] suf_{l+1}[b]) with
// pre_{l-1} = A_1 ... A_{l-1} (a row) and suf_{l+1} = A_{l+1} ... A_d (a
// column), inverse-transformed at the forward length (outputs 1..N do not
// alias). Every core entry (l, a, b) gets its own cotangent, also entries the
// plan stores no vector for (zero vectors, whose entries still have
// derivatives), through an entry table: entry e of an order is the core
// layout's position off_l + a R_l + b, its vector vid[e] or -1.
// Loss: with M_l = sum_i n_i H^(l)(i) and Z_l = sum_i g_i n_i H^(l)(i), for
// entry (l, a, b) coef = -1/(d-1)! w_l left_{l-1}[a] right_{l+1}[b] (the M
// chain) and sigma = -1/(d-1)! sum_{pos != l} w_pos pre[a] suf[b] of the chain
// with Z_pos in place of M_pos; then, as for CP,
//   gn_k = g_k sum_e coef_e h_e(k) + sum_e h_e(k) (ga_e(k) + sigma_e),
//   gH_e(k) = n_k (ga_e(k) + sigma_e) + coef_e g_k n_k.
#pragma once

#include "fft_kernels.cuh"
#include "vjp_kernels.cuh"

namespace sag {

// ---- spectrum of g from its column pass (scratch2): the rows of one row pair,
// split into the real spectrum in place; its Nyquist value into s_nyq.
template <class C>
__global__ void __launch_bounds__(kThreads) k_rows_tt_g(const __grid_constant__ RhsParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int j = find_segment(P.rowpre, P.nitems, blockIdx.x);
  const int oi = P.rowperm[j];
  const OrderDesc& od = P.ord[oi];
  const int kp = blockIdx.x - P.rowpre[j];
  const int M1 = od.M1, M2 = od.M2, ld = od.ld2;
  const int k1a = kp, k1b = M1 - kp;
  const int nrow = (kp == 0 || 2 * kp == M1) ? 1 : 2;
  const int NP = nrow * M2;
  C* buf1 = buf + 2 * ld;
  C* tw = buf1 + 2 * ld;
  const C* tw2 = static_cast<const C*>(od.tw2);
  const C* twL = static_cast<const C*>(od.twL);
  C* spec = static_cast<C*>(P.scratch2) + od.scr2_off;
  for (int i = threadIdx.x; i < M2; i += kThreads) tw[i] = tw2[i];
  for (int p = threadIdx.x; p < NP; p += kThreads) {
    const int row = p / M2, pos = p - row * M2;
    buf[row * ld + pos] = spec[(int64_t)(row ? k1b : k1a) * M2 + pos];
  }
  __syncthreads();
  C* res = fft_batch(buf, buf1, M2, ld, nrow, od.rp2, tw);
  for (int p = threadIdx.x; p < NP; p += kThreads) {
    const int row = p / M2, pos = p - row * M2;
    const int k1 = row ? k1b : k1a;
    int mrow, mpos;
    mirror_of(k1, row, pos, M1, M2, mrow, mpos);
    spec[(int64_t)k1 * M2 + pos] = unpack2(res[row * ld + pos], res[mrow * ld + mpos], twL[k1 + M1 * pos]);
    if (k1 == 0 && pos == 0) {
      const C z0 = res[0];
      const C zc = c_conj(z0);
      static_cast<C*>(P.s_nyq)[oi] = c_add(c_add(z0, zc), c_mul_pi(c_sub(z0, zc)));  // 2 G[M]
    }
  }
}

// ---- per frequency: every entry's cotangent spectrum G conj(pre[a] suf[b]).
// Thread e < M handles spectrum slot e, e = M the Nyquist value.
template <class C, int RMAX>
__global__ void __launch_bounds__(256) k_tt_chain_vjp(const __grid_constant__ RhsParams P) {
  const int oi = find_segment(P.chainpre, P.nitems, blockIdx.x);
  const OrderDesc& od = P.ord[oi];
  const int e = (blockIdx.x - P.chainpre[oi]) * blockDim.x + threadIdx.x;
  const int M = od.M, d = od.d;
  if (e > M) return;
  const C* spec = static_cast<const C*>(P.scratch) + od.scr_off;
  const C* nyq = static_cast<const C*>(P.spec_nyq);
  const int* vid = P.vid + od.vid_off;
  auto load = [&](int j) -> C {  // core entry j of the order, its vector vid[j] >= 0
    const int v = vid[j];
    const C z = (e < M) ? spec[(int64_t)(v - od.vbase) * M + e] : nyq[v];
    return tt_weight(z, P, od.vid_off + j);
  };
  const C G = (e < M) ? static_cast<const C*>(P.scratch2)[od.scr2_off + e] : static_cast<const C*>(P.s_nyq)[oi];
  C* out = static_cast<C*>(P.ent_spec) + od.ent_spec_off;
  C* out_nyq = static_cast<C*>(P.ent_nyq) + od.ebase;
  // prefixes pre_l = A_1 ... A_l (rows of length R_l), l = 0..d-1
  C pre[kMaxD][RMAX];
  pre[0][0] = c_one(C{});
  int off = 0;
  int offl[kMaxD + 1];
  for (int l = 1; l <= d; ++l) {
    offl[l] = off;
    const int ra = od.ttr[l - 1], rb = od.ttr[l];
    if (l < d) {
      for (int b = 0; b < rb; ++b) {
        C acc = c_zero(C{});
        for (int a = 0; a < ra; ++a) {
          const int j = off + a * rb + b;
          if (vid[j] >= 0) acc = c_add(acc, c_mul(pre[l - 1][a], load(j)));
        }
        pre[l][b] = acc;
      }
    }
    off += ra * rb;
  }
  // back through the cores with the suffix suf = A_{l+1} ... A_d (column of length R_l)
  C suf[RMAX], sn[RMAX];
  suf[0] = c_one(C{});
  for (int l = d; l >= 1; --l) {
    const int ra = od.ttr[l - 1], rb = od.ttr[l];
    for (int a = 0; a < ra; ++a)
      for (int b = 0; b < rb; ++b) {
        const int loc = offl[l] + a * rb + b;
        const C h = c_mul(G, c_conj(c_mul(pre[l - 1][a], suf[b])));
        if (e < M) out[(int64_t)loc * M + e] = h;
        else out_nyq[loc] = h;
      }
    if (l > 1) {
      for (int a = 0; a < ra; ++a) {
        C acc = c_zero(C{});
        for (int b = 0; b < rb; ++b) {
          const int j = offl[l] + a * rb + b;
          if (vid[j] >= 0) acc = c_add(acc, c_mul(load(j), suf[b]));
        }
        sn[a] = acc;
      }
      for (int a = 0; a < ra; ++a) suf[a] = sn[a];
    }
  }
}

// ---- inverse row half of every entry's cotangent spectrum (row pair of an
// order), in place, as the forward pass's inverse rows do for S.
template <class C>
__global__ void __launch_bounds__(kThreads) k_rows_tt_inv_vjp(const __grid_constant__ RhsParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int j = find_segment(P.rowpre, P.nitems, blockIdx.x);
  const int oi = P.rowperm[j];
  const OrderDesc& od = P.ord[oi];
  const int kp = blockIdx.x - P.rowpre[j];
  const int M1 = od.M1, M2 = od.M2, M = od.M, ld = od.ld2;
  const int k1a = kp, k1b = M1 - kp;
  const int nrow = (kp == 0 || 2 * kp == M1) ? 1 : 2;
  const int NP = nrow * M2;
  C* sS = buf;               // NP staged spectrum values
  C* bufa = buf + 2 * ld;    // two transform slots
  C* bufb = bufa + 2 * ld;
  C* tw = bufb + 2 * ld;
  const C* tw2 = static_cast<const C*>(od.tw2);
  const C* twL = static_cast<const C*>(od.twL);
  const C* tw4 = static_cast<const C*>(od.tw4);
  for (int i = threadIdx.x; i < M2; i += kThreads) tw[i] = tw2[i];
  for (int q = 0; q < od.nent; ++q) {
    C* S = static_cast<C*>(P.ent_spec) + od.ent_spec_off + (int64_t)q * M;
    const C SM = static_cast<const C*>(P.ent_nyq)[od.ebase + q];
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
    for (int p = threadIdx.x; p < NP; p += kThreads) {
      const int row = p / M2, j2 = p - row * M2;
      const int k1 = row ? k1b : k1a;
      S[(int64_t)k1 * M2 + j2] = c_mul(res[row * ld + j2], tw4[j2 * k1]);
    }
    __syncthreads();
  }
}

// ---- inverse column pass of every entry: its cotangent ga_e (FP64, sizes
// 1..N at eoff[e]), scaled back from the double-word path's exponents.
template <class C>
__global__ void __launch_bounds__(kThreads) k_inv_col_vjp_tt(const __grid_constant__ RhsParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int it = find_segment(P.entpre, P.nitems, blockIdx.x);
  const OrderDesc& od = P.ord[it];
  const int local = blockIdx.x - P.entpre[it];
  const int q = local / od.ncolblk, cb = local - q * od.ncolblk;
  const int W = od.W, M1 = od.M1, M2 = od.M2, ld = od.ld1, N = od.N;
  C* buf1 = buf + W * ld;
  C* tw = buf1 + W * ld;
  const C* tw1 = static_cast<const C*>(od.tw1);
  for (int i = threadIdx.x; i < M1; i += kThreads) tw[i] = tw1[i];
  const C* src = static_cast<const C*>(P.ent_spec) + od.ent_spec_off + (int64_t)q * od.M;
  for (int e = threadIdx.x; e < W * M1; e += kThreads) {
    const int c = e % W, k1 = e / W;
    buf[c * ld + k1] = src[(int64_t)k1 * M2 + cb * W + c];
  }
  __syncthreads();
  C* res = fft_batch(buf, buf1, M1, ld, W, od.rp1, tw);
  const int ge = od.ebase + q;
  const SysScalars& sc = P.sc[od.sys];
  const int ex = P.dwpath ? sc.e_g + P.eexcl[ge] + (od.d - 1) * sc.e_n : 0;
  const double scale = ldexp(od.gscale, ex);
  double* out = P.gaent + P.eoff[ge];
  for (int e = threadIdx.x; e < W * M1; e += kThreads) {
    const int c = e % W, j1 = e / W;
    const int jj = M2 * j1 + cb * W + c;
    const C w = res[c * ld + j1];
    const int k = 2 * jj;
    if (k >= 1 && k <= N) out[k - 1] = cre(w) * scale;
    if (k + 1 <= N) out[k] = -cim(w) * scale;
  }
}

// The TT adjoint's FFT stage after the vectors' forward columns: their row
// spectra, g's spectrum, every entry's cotangent spectrum, its inverse rows
// and its inverse columns (into gaent).
template <class C>
cudaError_t launch_vjp_tt_after_cols(const RhsParams& P, const LaunchCfg& L, const double* g, cudaStream_t st) {
  if (L.row_blocks == 0) return cudaGetLastError();  // every order idle: no cotangent spectra
  k_rows_tt_fwd<C><<<L.row_blocks, kThreads, L.rowtt_smem, st>>>(P);
  k_gcol<C><<<L.inv_blocks, kThreads, L.vcol_smem, st>>>(P, g);
  k_rows_tt_g<C><<<L.row_blocks, kThreads, L.rowtt_smem, st>>>(P);
  if (P.tt_rmax <= 4) k_tt_chain_vjp<C, 4><<<L.chain_blocks, 256, 0, st>>>(P);
  else if (P.tt_rmax <= 8) k_tt_chain_vjp<C, 8><<<L.chain_blocks, 256, 0, st>>>(P);
  else k_tt_chain_vjp<C, 16><<<L.chain_blocks, 256, 0, st>>>(P);
  k_rows_tt_inv_vjp<C><<<L.row_blocks, kThreads, L.rowtt_smem, st>>>(P);
  if (L.ent_blocks > 0) k_inv_col_vjp_tt<C><<<L.ent_blocks, kThreads, L.vcol_smem, st>>>(P);
  return cudaGetLastError();
}

template <class C>
cudaError_t setup_vjp_tt(const LaunchCfg& L) {
  (void)L;
  cudaError_t e = allow_max_smem(k_rows_tt_fwd<C>);  // this file's own copy (see allow_max_smem)
  if (e == cudaSuccess) e = allow_max_smem(k_rows_tt_g<C>);
  if (e == cudaSuccess) e = allow_max_smem(k_rows_tt_inv_vjp<C>);
  if (e == cudaSuccess) e = allow_max_smem(k_inv_col_vjp_tt<C>);
  return e;
}

}  // namespace sag
