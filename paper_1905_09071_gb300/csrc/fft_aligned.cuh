// Grid-aligned double-word butterflies (radix 2, 3, 4, 6 and 8) for the FFT
// passes.
//
// Most of a double-word butterfly's work is additions, and an error-free
// double-word addition costs eight float operations (TwoSum on the high words,
// then the low words). These butterflies first round the high words of their
// R (twiddled) inputs to one grid of spacing q, chosen from the largest input
// component, so that every sum and difference of the butterfly is exact in the
// high word and an addition costs two float operations: the exact sum of the
// high words and the rounded sum of the low words.
//
// The grid. Let m be the largest |real| or |imaginary| high word of the R
// inputs and e its binary exponent (m < 2^(e+1)). Each input, and each input
// times a unit twiddle, has modulus below sqrt2 2^(e+1); a radix-R DFT (R <= 8)
// adds at most R of them, so every intermediate and output component stays
// below 8 sqrt2 2^(e+1) < 2^(e+5). With q = 2^(e-19), every multiple of q below
// 2^24 q = 2^(e+5) is a float, so sums and differences of grid values are
// exact. (Radix 3 also halves a sum, exactly, onto the grid q/2; its values
// stay below 3 sqrt2 2^(e+1) < 2^(e+4) = 2^24 q/2. Radix 6, two radix-3 DFTs
// combined by sums and differences, reaches 6 sqrt2 2^(e+1) on that half
// grid, so it rounds to the grid 2q: values below 2^24 q = 2^(e+5).) A value v with |v| <= 2^22 q is rounded to the grid by one addition of
// the constant C = 1.5 2^23 q (v + C lies in [2^23 q, 2^24 q), whose float
// spacing is q) and one subtraction of C; with an FMA the product x y is
// rounded to the grid directly, and a second FMA gives its remainder
// x y - grid(x y) (|.| <= q/2), which joins the low word. The radix-8
// rotations by (1 -/+ i)/sqrt2 round to the same grid.
//
// Precision. A low word holds what lies below the grid (a few q) and rounds
// at 2^-24 of its size: about 2^-40 of the butterfly's largest input, against
// about 2^-47 of each value for the double-word operations of dw.cuh. The
// exactness argument uses the high words only; a low word larger than the grid
// (a value that shrank since the previous pass) is simply carried, rounding
// at its own 2^-24. The outputs are (grid high word, low word) pairs, which
// every other double-word operation accepts.
//
// Valid for |components| below 2^123 (the grid constant's exponent must not
// overflow); the FFT inputs are scaled to magnitudes near 1.
//
// Included by fft.cuh after its small-DFT constants, which it uses.
#pragma once

#include <stdint.h>
#include <string.h>

#include "dw.cuh"

namespace sag {

SAG_HD float f_amax(float a, float b) { return fmaxf(fabsf(a), fabsf(b)); }

// C = 1.5 * 2^(e + 4) for the binary exponent e of m (m >= 0): the grid
// q = 2^(e - 19). For m = 0 or subnormal m the grid is 2^-146.
SAG_HD float grid_const(float m) {
  uint32_t b;
#if defined(__CUDA_ARCH__)
  b = __float_as_uint(m);
#else
  memcpy(&b, &m, sizeof b);
#endif
  b = ((b & 0x7f800000u) + (4u << 23)) | 0x00400000u;
  float c;
#if defined(__CUDA_ARCH__)
  c = __uint_as_float(b);
#else
  memcpy(&c, &b, sizeof c);
#endif
  return c;
}

// Pair (a, b) (value a + b) with its high word rounded to the grid of C.
SAG_HD void g_snap(float a, float b, float C, float& h, float& l) {
  h = F_SUB(F_ADD(a, C), C);
  l = F_ADD(F_SUB(a, h), b);  // a - h is exact
}

// (h + l) (kh + kl) on the grid of C.
SAG_HD void g_kmul(float h, float l, float kh, float kl, float C, float& H, float& L) {
  H = F_SUB(F_FMA(h, kh, C), C);
  float r = F_FMA(h, kh, -H);
  r = F_FMA(h, kl, r);
  L = F_FMA(l, kh, r);
}

// x1 y1 + x2 y2 on the grid of C, for pairs x (high word on any grid) and
// double-word y; a difference passes -x2.
SAG_HD void g_dot2(float x1h, float x1l, float y1h, float y1l, float x2h, float x2l, float y2h, float y2l,
                   float C, float& H, float& L) {
  const float H1 = F_SUB(F_FMA(x1h, y1h, C), C);
  const float H2 = F_SUB(F_FMA(x2h, y2h, C), C);
  const float r1 = F_FMA(x1h, y1h, -H1);
  const float r2 = F_FMA(x2h, y2h, -H2);
  H = F_ADD(H1, H2);  // exact: both on the grid
  float t = F_ADD(r1, r2);
  t = F_FMA(x1h, y1l, t);
  t = F_FMA(x2h, y2l, t);
  t = F_FMA(x1l, y1h, t);
  L = F_FMA(x2l, y2h, t);
}

SAG_HD cdw g_cmul(cdw a, cdw w, float C) {
  cdw o;
  g_dot2(a.rh, a.rl, w.rh, w.rl, -a.ih, -a.il, w.ih, w.il, C, o.rh, o.rl);
  g_dot2(a.rh, a.rl, w.ih, w.il, a.ih, a.il, w.rh, w.rl, C, o.ih, o.il);
  return o;
}

SAG_HD cdw g_snapc(cdw a, float C) {
  cdw o;
  g_snap(a.rh, a.rl, C, o.rh, o.rl);
  g_snap(a.ih, a.il, C, o.ih, o.il);
  return o;
}

// Sums of grid pairs: exact high words, rounded low words.
SAG_HD cdw g_add(cdw a, cdw b) {
  return cdw{F_ADD(a.rh, b.rh), F_ADD(a.rl, b.rl), F_ADD(a.ih, b.ih), F_ADD(a.il, b.il)};
}
SAG_HD cdw g_sub(cdw a, cdw b) {
  return cdw{F_SUB(a.rh, b.rh), F_SUB(a.rl, b.rl), F_SUB(a.ih, b.ih), F_SUB(a.il, b.il)};
}

// a omega_8 = (re + im, im - re) / sqrt2 and a omega_8^3 = (im - re, -(re + im)) / sqrt2,
// omega_8 = exp(-i pi / 4); the sums are exact, the scaling rounds to the grid.
template <bool THREE>
SAG_HD cdw g_rot8(cdw a, float C) {
  const float sh = F_ADD(a.rh, a.ih), sl = F_ADD(a.rl, a.il);
  const float dh = F_SUB(a.ih, a.rh), dl = F_SUB(a.il, a.rl);
  cdw o;
  if constexpr (!THREE) {
    g_kmul(sh, sl, K_SQRT1_2.hi, K_SQRT1_2.lo, C, o.rh, o.rl);
    g_kmul(dh, dl, K_SQRT1_2.hi, K_SQRT1_2.lo, C, o.ih, o.il);
  } else {
    g_kmul(dh, dl, K_SQRT1_2.hi, K_SQRT1_2.lo, C, o.rh, o.rl);
    g_kmul(sh, sl, -K_SQRT1_2.hi, -K_SQRT1_2.lo, C, o.ih, o.il);
  }
  return o;
}

SAG_HD void g_dft4v(cdw y0, cdw y1, cdw y2, cdw y3, cdw& Y0, cdw& Y1, cdw& Y2, cdw& Y3) {
  const cdw s0 = g_add(y0, y2), s1 = g_sub(y0, y2);
  const cdw s2 = g_add(y1, y3), s3 = c_mul_mi(g_sub(y1, y3));
  Y0 = g_add(s0, s2);
  Y2 = g_sub(s0, s2);
  Y1 = g_add(s1, s3);
  Y3 = g_sub(s1, s3);
}

// The same splittings as dft2/dft3/dft4/dft6/dft8 of fft.cuh, on grid pairs.
template <int R>
SAG_HD void g_dft(cdw* x, float C) {
  if constexpr (R == 3) {
    const cdw t1 = g_add(x[1], x[2]);
    const cdw t2 = g_sub(x[0], c_scale2(t1, 0.5f));
    const cdw d = g_sub(x[1], x[2]);
    cdw t3;  // -i (x1 - x2) sqrt3/2
    g_kmul(d.ih, d.il, K_SQRT3_2.hi, K_SQRT3_2.lo, C, t3.rh, t3.rl);
    g_kmul(d.rh, d.rl, -K_SQRT3_2.hi, -K_SQRT3_2.lo, C, t3.ih, t3.il);
    x[0] = g_add(x[0], t1);
    x[1] = g_add(t2, t3);
    x[2] = g_sub(t2, t3);
  } else if constexpr (R == 6) {  // prime-factor split, as dft6 of fft.cuh
    cdw y0[3] = {x[0], x[2], x[4]}, y1[3] = {x[3], x[5], x[1]};
    g_dft<3>(y0, C);
    g_dft<3>(y1, C);
    x[0] = g_add(y0[0], y1[0]);
    x[3] = g_sub(y0[0], y1[0]);
    x[4] = g_add(y0[1], y1[1]);
    x[1] = g_sub(y0[1], y1[1]);
    x[2] = g_add(y0[2], y1[2]);
    x[5] = g_sub(y0[2], y1[2]);
  } else if constexpr (R == 2) {
    const cdw a = x[0], b = x[1];
    x[0] = g_add(a, b);
    x[1] = g_sub(a, b);
  } else if constexpr (R == 4) {
    g_dft4v(x[0], x[1], x[2], x[3], x[0], x[1], x[2], x[3]);
  } else {
    static_assert(R == 8, "grid butterflies exist for radix 2, 3, 4, 6 and 8");
    const cdw a0 = g_add(x[0], x[4]), b0 = g_sub(x[0], x[4]);
    const cdw a1 = g_add(x[1], x[5]), b1 = g_rot8<false>(g_sub(x[1], x[5]), C);
    const cdw a2 = g_add(x[2], x[6]), b2 = c_mul_mi(g_sub(x[2], x[6]));
    const cdw a3 = g_add(x[3], x[7]), b3 = g_rot8<true>(g_sub(x[3], x[7]), C);
    g_dft4v(a0, a1, a2, a3, x[0], x[2], x[4], x[6]);
    g_dft4v(b0, b1, b2, b3, x[1], x[3], x[5], x[7]);
  }
}

// Largest |component| of the high words of x[0..R), as a balanced tree.
template <int R>
SAG_HD float g_maxabs(const cdw* x) {
  float m[R];
#pragma unroll
  for (int t = 0; t < R; ++t) m[t] = f_amax(x[t].rh, x[t].ih);
  if constexpr (R == 3) {
    return fmaxf(m[0], fmaxf(m[1], m[2]));
  } else if constexpr (R == 6) {
    return fmaxf(fmaxf(fmaxf(m[0], m[3]), fmaxf(m[1], m[4])), fmaxf(m[2], m[5]));
  } else {
#pragma unroll
    for (int w = R / 2; w >= 1; w /= 2)
#pragma unroll
      for (int t = 0; t < w; ++t) m[t] = fmaxf(m[t], m[t + w]);
    return m[0];
  }
}

template <int R>
inline constexpr bool g_radix = R == 2 || R == 3 || R == 4 || R == 6 || R == 8;

// Radix-R butterfly: inputs t >= 1 multiplied by tw(t) when TW, then the DFT,
// in grid arithmetic.
template <int R, bool TW, class TWF>
SAG_HD void g_bfly(cdw* x, TWF tw) {
  // radix 6: one grid step coarser (constant 2 C), see the header
  const float C = grid_const(g_maxabs<R>(x)) * (R == 6 ? 2.0f : 1.0f);
  x[0] = g_snapc(x[0], C);
#pragma unroll
  for (int t = 1; t < R; ++t) {
    if constexpr (TW) x[t] = g_cmul(x[t], tw(t), C);
    else x[t] = g_snapc(x[t], C);
  }
  g_dft<R>(x, C);
}

}  // namespace sag
