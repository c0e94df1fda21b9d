// Double-word power u i^a of the parametric factors U(i) = u i^a, generated
// where the forward FFT needs them instead of being read from memory.
//
// i^a = exp(a ln i) with ln i from a per-plan table (double-word, one entry
// per size) and exp by the table-driven method of P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM Trans. Math. Softw. 15(2), 1989, carried out in
// double-word arithmetic:
//   t = a ln i;  k = nearest integer to t 64/ln 2,  k = 64 m + j (0 <= j < 64);
//   r = t - k ln2/64  (|r| <= ln2/128, Cody-Waite reduction with ln2/64 split
//       into c1 + c2 + c3, c1 short enough that k c1 is exact);
//   exp(t) = 2^m 2^(j/64) exp(r),  exp(r) by its Taylor polynomial to r^5
//       (the r^6 term is below 2^-53), the low orders in double-word.
// The split constants and the 64 values 2^(j/64) are computed on the host from
// the long-double logarithm and exp2 (make_exp_consts); nothing here is a
// stored library constant.
//
// Accuracy: the argument t carries the double-word rounding of a ln i, about
// 2^-47 |t|, which exp turns into a relative error; the reduction, the
// polynomial and the table add a few 2^-48. For |t| <= 8 the result is within
// about 1e-13 relative of u i^a (checked against a long-double power over all
// i <= 2^22 on the host, and on the device through sag_power_eval).
#pragma once

#include <cmath>

#include "dw.cuh"

namespace sag {

// [0] 64/ln2, [1..3] c1, c2, c3 with c1 + c2 + c3 = ln2/64 (c1 has 12
// significant bits, so k c1 is exact for |k| < 4096), [4 + 2j], [5 + 2j] the
// double-word 2^(j/64), j < 64.
constexpr int kExpConsts = 4 + 128;

inline void make_exp_consts(float* out) {
  const long double step = logl(2.0L) / 64.0L;
  out[0] = (float)(1.0L / step);
  int e = 0;
  std::frexp((double)step, &e);
  const long double c1 = ldexpl(nearbyintl(ldexpl(step, 12 - e)), e - 12);
  const float c2 = (float)(step - c1);
  const float c3 = (float)(step - c1 - (long double)c2);
  out[1] = (float)c1;
  out[2] = c2;
  out[3] = c3;
  for (int j = 0; j < 64; ++j) {
    const long double t = exp2l((long double)j / 64.0L);
    const float hi = (float)t;
    out[4 + 2 * j] = hi;
    out[5 + 2 * j] = (float)(t - hi);
  }
}

#if defined(__CUDA_ARCH__)
#define SAG_RINT(x) rintf(x)
#define SAG_LDG(p) __ldg(p)
#else
#define SAG_RINT(x) std::nearbyint(x)
#define SAG_LDG(p) (*(p))
#endif

// 2^m as a float for |m| <= 126 (exact).
SAG_HD float pow2f(int m) {
  union {
    unsigned u;
    float f;
  } x;
  x.u = (unsigned)(m + 127) << 23;
  return x.f;
}

// exp(t) for a double-word t with |t| < 44.
SAG_HD dw dw_exp(dw t, const float* __restrict__ ek) {
  const float kf = SAG_RINT(F_MUL(t.hi, SAG_LDG(ek)));
  const int k = (int)kf;
  const int m = k >> 6, j = k & 63;  // floor division: k = 64 m + j
  // r = t - k (c1 + c2 + c3): k c1 is exact, and so are the differences
  // formed with TwoSum and the product k c2 formed with TwoProd; the low
  // terms are summed in FP32 (they are about 2^-24 of r).
  float a1, a1e;
  two_sum(t.hi, -F_MUL(kf, SAG_LDG(ek + 1)), a1, a1e);
  const float p2 = F_MUL(kf, SAG_LDG(ek + 2));
  const float p2e = F_FMA(kf, SAG_LDG(ek + 2), -p2);
  float sh, sl;
  two_sum(a1, -p2, sh, sl);
  sl = F_ADD(F_ADD(sl, a1e), F_SUB(F_SUB(t.lo, p2e), F_MUL(kf, SAG_LDG(ek + 3))));
  dw r;
  fast_two_sum(sh, sl, r.hi, r.lo);
  // exp(r) = 1 + r (1 + r (1/2 + r (1/6 + r (1/24 + r/120)))): the two inner
  // levels in FP32 (their error is scaled by r^3 <= 2^-22), the rest in
  // double-word.
  const float c4 = F_FMA(r.hi, 1.0f / 120.0f, 1.0f / 24.0f);
  const float c3 = F_FMA(r.hi, c4, 1.0f / 6.0f);
  const float q = F_MUL(r.hi, c3);
  dw s;
  two_sum(0.5f, q, s.hi, s.lo);
  s = dw_mul(r, s);
  float h, l;
  two_sum(1.0f, s.hi, h, l);
  s = dw{h, F_ADD(l, s.lo)};
  s = dw_mul(r, s);
  two_sum(1.0f, s.hi, h, l);
  s = dw{h, F_ADD(l, s.lo)};
  const dw tj{SAG_LDG(ek + 4 + 2 * j), SAG_LDG(ek + 5 + 2 * j)};
  return dw_scale2(dw_mul(s, tj), pow2f(m));
}

// u i^a from (u, a) as double-words and ln i (double-word).
SAG_HD dw dw_power(dw u, dw a, dw lni, const float* __restrict__ ek) {
  return dw_mul(u, dw_exp(dw_mul(a, lni), ek));
}

}  // namespace sag
