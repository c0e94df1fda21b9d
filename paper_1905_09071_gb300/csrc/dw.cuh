// Double-word ("float-float") arithmetic and the two complex scalar types the
// FFT path is templated on.
//
// A dw value is the unevaluated sum hi + lo of two floats, about 48 significant
// bits. The building blocks are the error-free transforms of Dekker (1971) and
// Knuth (TAOCP vol. 2, Sec. 4.2.2): TwoSum, Fast2Sum, and the FMA-based
// TwoProd; the composite operations follow the "sloppy" addition and FMA
// multiplication analysed by Joldes, Muller and Popescu (2017), whose error is
// bounded relative to |a| + |b| (resp. |a||b|), which is what a normwise FFT
// error bound needs.
//
// Conversions from FP64 produce normalised pairs (|lo| <= ulp(hi)/2). The
// arithmetic operations leave their result unnormalised: the final Fast2Sum
// that would fold the error word into hi is skipped. That keeps every leading
// sum and product error-free (TwoSum and TwoProd do not need normalised
// inputs), and the error word only collects the rounding errors of the
// leading operations plus the low words of the operands, each at most about
// 2^-24 times the operands' magnitudes; the terms a normalised version would
// add or drop are of the order 2^-48 |a| |b| (products) or 2^-48 (|a| + |b|)
// (sums) as well. The error bounds stay normwise with a unit of about 2^-47
// instead of 2^-48, for three FP32 operations fewer per addition and per
// product.
//
// Every float operation below is written with an explicit round-to-nearest
// intrinsic so the compiler can neither contract nor reassociate it; the
// error-free transforms are only exact that way.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#if defined(__CUDA_ARCH__)
#define SAG_HD __host__ __device__ __forceinline__
#define F_ADD(a, b) __fadd_rn((a), (b))
#define F_SUB(a, b) __fsub_rn((a), (b))
#define F_MUL(a, b) __fmul_rn((a), (b))
#define F_FMA(a, b, c) __fmaf_rn((a), (b), (c))
#else
// Host build of the same code (used by host-side unit checks); requires
// -ffp-contract=off so that a + b and a * b stay separately rounded.
#define SAG_HD inline
#define F_ADD(a, b) ((a) + (b))
#define F_SUB(a, b) ((a) - (b))
#define F_MUL(a, b) ((a) * (b))
#define F_FMA(a, b, c) fmaf((a), (b), (c))
#endif

namespace sag {

struct dw {
  float hi, lo;
};

struct __align__(16) cdw {
  float rh, rl, ih, il;  // re = rh + rl, im = ih + il
};

// The same double-word complex value for the path whose FFT butterflies all
// run in the double-word operations below (cdw's radix-2/3/4/8 butterflies are
// grid-aligned, fft_aligned.cuh). A distinct type so that the two paths'
// kernels are distinct instantiations; every cdw operation applies to it and
// converts back.
struct __align__(16) cdwx : cdw {
  cdwx() = default;
  SAG_HD cdwx(const cdw& a) : cdw(a) {}
};
static_assert(sizeof(cdwx) == sizeof(cdw), "cdwx shares cdw's layout");

template <class C> struct is_dw : std::false_type {};
template <> struct is_dw<cdw> : std::true_type {};
template <> struct is_dw<cdwx> : std::true_type {};

struct __align__(16) cd {
  double re, im;
};

// ---- error-free transforms --------------------------------------------------
SAG_HD void two_sum(float a, float b, float& s, float& e) {
  s = F_ADD(a, b);
  float bb = F_SUB(s, a);
  e = F_ADD(F_SUB(a, F_SUB(s, bb)), F_SUB(b, bb));
}
SAG_HD void fast_two_sum(float a, float b, float& s, float& e) {
  s = F_ADD(a, b);
  e = F_SUB(b, F_SUB(s, a));
}

// ---- real double-word -------------------------------------------------------
SAG_HD dw dw_add(dw a, dw b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = F_ADD(e, F_ADD(a.lo, b.lo));
  return dw{s, e};
}
SAG_HD dw dw_neg(dw a) { return dw{-a.hi, -a.lo}; }
SAG_HD dw dw_sub(dw a, dw b) { return dw_add(a, dw_neg(b)); }
SAG_HD dw dw_mul(dw a, dw b) {
  float p = F_MUL(a.hi, b.hi);
  float e = F_FMA(a.hi, b.hi, -p);
  e = F_FMA(a.hi, b.lo, e);
  e = F_FMA(a.lo, b.hi, e);
  return dw{p, e};
}
// a * 2^k for a power-of-two float scale (exact unless it under/overflows).
SAG_HD dw dw_scale2(dw a, float p2) { return dw{F_MUL(a.hi, p2), F_MUL(a.lo, p2)}; }

// Split of a double into a double-word (exact when the double has <= 48
// significant bits, otherwise rounded to nearest in the low word).
SAG_HD dw dw_from_double(double x) {
  float hi = (float)x;
  float lo = (float)(x - (double)hi);
  return dw{hi, lo};
}
SAG_HD double dw_to_double(dw a) { return (double)a.hi + (double)a.lo; }

// ---- complex double-word ----------------------------------------------------
SAG_HD cdw make_cdw(dw re, dw im) { return cdw{re.hi, re.lo, im.hi, im.lo}; }
SAG_HD dw re_of(cdw a) { return dw{a.rh, a.rl}; }
SAG_HD dw im_of(cdw a) { return dw{a.ih, a.il}; }

SAG_HD cdw c_add(cdw a, cdw b) { return make_cdw(dw_add(re_of(a), re_of(b)), dw_add(im_of(a), im_of(b))); }
SAG_HD cdw c_sub(cdw a, cdw b) { return make_cdw(dw_sub(re_of(a), re_of(b)), dw_sub(im_of(a), im_of(b))); }
SAG_HD cdw c_conj(cdw a) { return cdw{a.rh, a.rl, -a.ih, -a.il}; }
// a * (-i) and a * (+i)
SAG_HD cdw c_mul_mi(cdw a) { return cdw{a.ih, a.il, -a.rh, -a.rl}; }
SAG_HD cdw c_mul_pi(cdw a) { return cdw{-a.ih, -a.il, a.rh, a.rl}; }
SAG_HD cdw c_scale2(cdw a, float p2) {
  return cdw{F_MUL(a.rh, p2), F_MUL(a.rl, p2), F_MUL(a.ih, p2), F_MUL(a.il, p2)};
}
SAG_HD cdw c_real_mul(cdw a, dw s) { return make_cdw(dw_mul(re_of(a), s), dw_mul(im_of(a), s)); }
SAG_HD cdw c_zero(cdw) { return cdw{0.f, 0.f, 0.f, 0.f}; }
SAG_HD cdw c_one(cdw) { return cdw{1.f, 0.f, 0.f, 0.f}; }

// One component of a complex product, x1*y1 - x2*y2 (sub = true) or
// x1*y1 + x2*y2: both leading products are formed exactly (TwoProd), their sum
// exactly (TwoSum), and the first-order cross terms are folded into the error
// word with FMAs.
SAG_HD dw dot2(dw x1, dw y1, dw x2, dw y2, bool sub) {
  float p1 = F_MUL(x1.hi, y1.hi);
  float e1 = F_FMA(x1.hi, y1.hi, -p1);
  float x2h = sub ? -x2.hi : x2.hi;
  float x2l = sub ? -x2.lo : x2.lo;
  float p2 = F_MUL(x2h, y2.hi);
  float e2 = F_FMA(x2h, y2.hi, -p2);
  float s, es;
  two_sum(p1, p2, s, es);
  float t = F_ADD(F_ADD(e1, e2), es);
  t = F_FMA(x1.hi, y1.lo, t);
  t = F_FMA(x1.lo, y1.hi, t);
  t = F_FMA(x2h, y2.lo, t);
  t = F_FMA(x2l, y2.hi, t);
  return dw{s, t};
}
SAG_HD cdw c_mul(cdw a, cdw b) {
  dw ar = re_of(a), ai = im_of(a), br = re_of(b), bi = im_of(b);
  return make_cdw(dot2(ar, br, ai, bi, true), dot2(ar, bi, ai, br, false));
}

// ---- complex double (FP64 path) --------------------------------------------
SAG_HD cd c_add(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
SAG_HD cd c_sub(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
SAG_HD cd c_conj(cd a) { return cd{a.re, -a.im}; }
SAG_HD cd c_mul_mi(cd a) { return cd{a.im, -a.re}; }
SAG_HD cd c_mul_pi(cd a) { return cd{-a.im, a.re}; }
SAG_HD cd c_scale2(cd a, float p2) { return cd{a.re * (double)p2, a.im * (double)p2}; }
SAG_HD cd c_real_mul(cd a, double s) { return cd{a.re * s, a.im * s}; }
SAG_HD cd c_zero(cd) { return cd{0.0, 0.0}; }
SAG_HD cd c_one(cd) { return cd{1.0, 0.0}; }
SAG_HD cd c_mul(cd a, cd b) {
#if defined(__CUDA_ARCH__)
  return cd{__fma_rn(a.re, b.re, -a.im * b.im), __fma_rn(a.re, b.im, a.im * b.re)};
#else
  return cd{fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
#endif
}

// Real scalar of each complex type, and conversions from FP64.
template <class C> struct real_of;
template <> struct real_of<cdw> { using type = dw; };
template <> struct real_of<cdwx> { using type = dw; };
template <> struct real_of<cd> { using type = double; };

SAG_HD void from_double(double x, dw& out) { out = dw_from_double(x); }
SAG_HD void from_double(double x, double& out) { out = x; }
SAG_HD cdw cfrom(double re, double im, cdw) { return make_cdw(dw_from_double(re), dw_from_double(im)); }
SAG_HD cd cfrom(double re, double im, cd) { return cd{re, im}; }
SAG_HD double cre(cdw a) { return (double)a.rh + (double)a.rl; }
SAG_HD double cim(cdw a) { return (double)a.ih + (double)a.il; }
SAG_HD double cre(cd a) { return a.re; }
SAG_HD double cim(cd a) { return a.im; }

}  // namespace sag
