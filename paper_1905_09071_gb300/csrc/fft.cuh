// Batched Stockham FFT building blocks, templated on the complex scalar (cd for
// FP64, cdw for double-word FP32).
//
// Forward transforms use omega_P = exp(-2 pi i / P). A length-P transform is a
// sequence of radix passes R_1, R_2, ... (product P). Pass number s with radix R
// and span Ns = R_1 ... R_{s-1} takes, for each butterfly j in [0, P/R), the
// inputs x[j + t P/R] (t < R), multiplies input t by omega_{Ns R}^{t (j mod Ns)},
// applies the radix-R DFT and writes output t to
//   (j / Ns) * Ns * R + (j mod Ns) + t * Ns,
// so that after the last pass the result is in natural order (Stockham's
// self-sorting formulation: no bit reversal, one out-of-place buffer swap per
// pass). The in-pass twiddle omega_{Ns R}^{e} is read as omega_P^{e P / (Ns R)}
// from one table of P entries.
#pragma once

#include <type_traits>

#include "dw.cuh"

namespace sag {

// ---- constants of the small DFTs, as (FP64, double-word) pairs ---------------
// hi/lo words are the float rounding of the constant and of its remainder.
struct kconst {
  double d;
  float hi, lo;
};
#define SAG_K(name, dv, h, l) constexpr kconst name = {dv, h, l};
SAG_K(K_SQRT1_2, 0.70710678118654752440, 7.071067691e-01f, 1.210161749e-08f)
SAG_K(K_SQRT3_2, 0.86602540378443864676, 8.660253882e-01f, 1.554362505e-08f)
SAG_K(K_C1_5, 0.30901699437494742410, 3.090170026e-01f, -8.207602598e-09f)
SAG_K(K_C2_5, -0.80901699437494742410, -8.090170026e-01f, 8.207602598e-09f)
SAG_K(K_S1_5, 0.95105651629515357212, 9.510565400e-01f, -2.371720598e-08f)
SAG_K(K_S2_5, 0.58778525229247312917, 5.877852440e-01f, 8.304436250e-09f)
#undef SAG_K

SAG_HD cd kmul(cd a, kconst k) { return c_real_mul(a, k.d); }
SAG_HD cdw kmul(cdw a, kconst k) { return c_real_mul(a, dw{k.hi, k.lo}); }
SAG_HD cd half(cd a) { return c_scale2(a, 0.5f); }
SAG_HD cdw half(cdw a) { return c_scale2(a, 0.5f); }

// ---- small DFTs in registers (forward) --------------------------------------
template <class C>
SAG_HD void dft2(C* x) {
  C a = x[0], b = x[1];
  x[0] = c_add(a, b);
  x[1] = c_sub(a, b);
}

template <class C>
SAG_HD void dft4v(C y0, C y1, C y2, C y3, C& Y0, C& Y1, C& Y2, C& Y3) {
  C s0 = c_add(y0, y2), s1 = c_sub(y0, y2);
  C s2 = c_add(y1, y3), s3 = c_mul_mi(c_sub(y1, y3));
  Y0 = c_add(s0, s2);
  Y2 = c_sub(s0, s2);
  Y1 = c_add(s1, s3);
  Y3 = c_sub(s1, s3);
}

template <class C>
SAG_HD void dft4(C* x) {
  dft4v(x[0], x[1], x[2], x[3], x[0], x[1], x[2], x[3]);
}

template <class C>
SAG_HD void dft8(C* x) {
  // Split n = j + 4t: even outputs are the DFT4 of a_j = x_j + x_{j+4}; odd
  // outputs the DFT4 of b_j omega_8^j with b_j = x_j - x_{j+4}.
  C a0 = c_add(x[0], x[4]), b0 = c_sub(x[0], x[4]);
  C a1 = c_add(x[1], x[5]), b1 = c_sub(x[1], x[5]);
  C a2 = c_add(x[2], x[6]), b2 = c_sub(x[2], x[6]);
  C a3 = c_add(x[3], x[7]), b3 = c_sub(x[3], x[7]);
  // b1 * omega_8 = b1 (1 - i)/sqrt2 ; b2 * (-i) ; b3 * omega_8^3 = b3 (-1 - i)/sqrt2
  b1 = kmul(c_add(b1, c_mul_mi(b1)), K_SQRT1_2);
  b2 = c_mul_mi(b2);
  b3 = kmul(c_sub(c_mul_mi(b3), b3), K_SQRT1_2);
  dft4v(a0, a1, a2, a3, x[0], x[2], x[4], x[6]);
  dft4v(b0, b1, b2, b3, x[1], x[3], x[5], x[7]);
}

template <class C>
SAG_HD void dft3(C* x) {
  C t1 = c_add(x[1], x[2]);
  C t2 = c_sub(x[0], half(t1));
  C t3 = c_mul_mi(kmul(c_sub(x[1], x[2]), K_SQRT3_2));
  x[0] = c_add(x[0], t1);
  x[1] = c_add(t2, t3);
  x[2] = c_sub(t2, t3);
}

template <class C>
SAG_HD void dft5(C* x) {
  C t1 = c_add(x[1], x[4]), t2 = c_add(x[2], x[3]);
  C t3 = c_sub(x[1], x[4]), t4 = c_sub(x[2], x[3]);
  C a1 = c_add(x[0], c_add(kmul(t1, K_C1_5), kmul(t2, K_C2_5)));
  C a2 = c_add(x[0], c_add(kmul(t1, K_C2_5), kmul(t2, K_C1_5)));
  C b1 = c_add(kmul(t3, K_S1_5), kmul(t4, K_S2_5));
  C b2 = c_sub(kmul(t3, K_S2_5), kmul(t4, K_S1_5));
  x[0] = c_add(x[0], c_add(t1, t2));
  x[1] = c_add(a1, c_mul_mi(b1));
  x[4] = c_sub(a1, c_mul_mi(b1));
  x[2] = c_add(a2, c_mul_mi(b2));
  x[3] = c_sub(a2, c_mul_mi(b2));
}

// Six points by the prime-factor split 6 = 2 x 3 (no internal twiddles):
// with n = (3 n1 + 2 n2) mod 6 the 3-point DFTs of (x0, x2, x4) and
// (x3, x5, x1) give Y0, Y1, and X[(3 k1 + 4 k2) mod 6] = Y0[k2] +- Y1[k2].
template <class C>
SAG_HD void dft6(C* x) {
  C y0[3] = {x[0], x[2], x[4]}, y1[3] = {x[3], x[5], x[1]};
  dft3(y0);
  dft3(y1);
  x[0] = c_add(y0[0], y1[0]);
  x[3] = c_sub(y0[0], y1[0]);
  x[4] = c_add(y0[1], y1[1]);
  x[1] = c_sub(y0[1], y1[1]);
  x[2] = c_add(y0[2], y1[2]);
  x[5] = c_sub(y0[2], y1[2]);
}

template <int R, class C>
SAG_HD void dft_r(C* x) {
  if constexpr (R == 2) dft2(x);
  else if constexpr (R == 3) dft3(x);
  else if constexpr (R == 4) dft4(x);
  else if constexpr (R == 5) dft5(x);
  else if constexpr (R == 6) dft6(x);
  else dft8(x);
}

}  // namespace sag

#include "fft_aligned.cuh"

namespace sag {

// One Stockham butterfly: transform-local index j of a length-P transform,
// pass radix R, span Ns. `in` and `out` point at the transform's first element.
// Double-word radix-2/3/4/8 butterflies run in grid-aligned arithmetic
// (fft_aligned.cuh).
template <int R, class C>
SAG_HD void stockham_bfly(const C* in, C* out, int P, int Ns, int j, const C* tw) {
  const int stride = P / R;
  const int k = j % Ns;
  const int twstep = P / (Ns * R);
  C x[R];
#pragma unroll
  for (int t = 0; t < R; ++t) x[t] = in[j + t * stride];
  if constexpr (std::is_same<C, cdw>::value && g_radix<R>) {
    auto twf = [&](int t) { return tw[t * k * twstep]; };
    if (Ns > 1) g_bfly<R, true>(x, twf);
    else g_bfly<R, false>(x, twf);
  } else {
    if (Ns > 1) {
#pragma unroll
      for (int t = 1; t < R; ++t) x[t] = c_mul(x[t], tw[t * k * twstep]);
    }
    dft_r<R>(x);
  }
  const int base = (j / Ns) * Ns * R + k;
#pragma unroll
  for (int t = 0; t < R; ++t) out[base + t * Ns] = x[t];
}

// Radix schedule of a length: odd radices first (3, 5), then as many 8s as
// possible, then one 4 or 2. Returns the number of passes (0 for P = 1), or -1
// if P has a prime factor other than 2, 3, 5 or a repeated 3 or 5.
struct radix_plan {
  int n;
  int r[16];
};
inline radix_plan make_radix_plan(int P) {
  radix_plan rp{};
  rp.n = 0;
  if (P % 3 == 0) { rp.r[rp.n++] = 3; P /= 3; }
  if (P % 5 == 0) { rp.r[rp.n++] = 5; P /= 5; }
  while (P % 8 == 0) {
    rp.r[rp.n++] = 8;
    P /= 8;
  }
  if (P == 4) { rp.r[rp.n++] = 4; P = 1; }
  if (P == 2) { rp.r[rp.n++] = 2; P = 1; }
  if (P != 1) rp.n = -1;
  return rp;
}

#if defined(__CUDACC__)
// Runs `count` independent length-P transforms stored in shared memory with a
// leading dimension ld >= P (transform b at buf + b * ld; ld = P + 1 spreads
// neighbouring transforms over different banks). Ping-pongs between buf0 and buf1 and
// returns the buffer holding the result. Every thread of the block must call
// it; it ends with a barrier.
template <class C>
__device__ C* fft_batch(C* buf0, C* buf1, int P, int ld, int count, const radix_plan& rp,
                        const C* tw) {
  C* in = buf0;
  C* out = buf1;
  int Ns = 1;
  for (int s = 0; s < rp.n; ++s) {
    const int R = rp.r[s];
    const int nb = P / R;
    const int total = nb * count;
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
      const int b = w / nb, j = w - b * nb;
      const C* ib = in + (size_t)b * ld;
      C* ob = out + (size_t)b * ld;
      switch (R) {
        case 8: stockham_bfly<8>(ib, ob, P, Ns, j, tw); break;
        case 4: stockham_bfly<4>(ib, ob, P, Ns, j, tw); break;
        case 2: stockham_bfly<2>(ib, ob, P, Ns, j, tw); break;
        case 3: stockham_bfly<3>(ib, ob, P, Ns, j, tw); break;
        default: stockham_bfly<5>(ib, ob, P, Ns, j, tw); break;
      }
    }
    __syncthreads();
    Ns *= R;
    C* t = in;
    in = out;
    out = t;
  }
  return in;
}
#endif

}  // namespace sag
