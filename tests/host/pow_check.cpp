// Host check of the double-word power u i^a of csrc/dw_pow.cuh: the same code
// compiled for the CPU (-ffp-contract=off keeps every FP32 operation separately
// rounded, as the device build's explicit intrinsics do) against a long-double
// power, for every size i = 1..N and each exponent given on the command line.
// Prints one line per exponent: a, the largest relative error, and the i where
// it occurs.
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "dw_pow.cuh"

int main(int argc, char** argv) {
  if (argc < 4) {
    std::fprintf(stderr, "usage: pow_check N u a1 [a2 ...]\n");
    return 2;
  }
  const int N = std::atoi(argv[1]);
  const double u = std::atof(argv[2]);
  float ek[sag::kExpConsts];
  sag::make_exp_consts(ek);
  for (int ai = 3; ai < argc; ++ai) {
    const double a = std::atof(argv[ai]);
    const sag::dw ad = sag::dw_from_double(a), ud = sag::dw_from_double(u);
    double worst = 0.0;
    int at = 0;
    for (int i = 1; i <= N; ++i) {
      const long double lni = logl((long double)i);
      const float lh = (float)lni;
      const sag::dw l{lh, (float)(lni - lh)};
      const sag::dw y = sag::dw_power(ud, ad, l, ek);
      const long double ref = (long double)u * expl((long double)a * lni);
      const double err = (double)fabsl(((long double)y.hi + (long double)y.lo - ref) / ref);
      if (err > worst) {
        worst = err;
        at = i;
      }
    }
    std::printf("%.17g %.3e %d\n", a, worst, at);
  }
  return 0;
}
