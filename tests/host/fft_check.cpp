// Host-side check of the library's FFT building blocks (csrc/dw.cuh, csrc/fft.cuh):
// runs the Stockham passes sequentially on the CPU for the FP64 and double-word
// complex types and prints, per length, the max-norm error relative to a
// long-double direct DFT. Compiled by tests/test_fft_host.py with
// -ffp-contract=off so that float operations stay separately rounded.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "fft.cuh"

using namespace sag;

template <class C>
static std::vector<C> stockham(std::vector<C> a, int P, const std::vector<C>& tw) {
  radix_plan rp = make_radix_plan(P);
  if (rp.n < 0) {
    std::printf("unsupported %d\n", P);
    std::exit(2);
  }
  std::vector<C> b(P);
  int Ns = 1;
  for (int s = 0; s < rp.n; ++s) {
    const int R = rp.r[s];
    for (int j = 0; j < P / R; ++j) {
      switch (R) {
        case 8: stockham_bfly<8>(a.data(), b.data(), P, Ns, j, tw.data()); break;
        case 4: stockham_bfly<4>(a.data(), b.data(), P, Ns, j, tw.data()); break;
        case 2: stockham_bfly<2>(a.data(), b.data(), P, Ns, j, tw.data()); break;
        case 3: stockham_bfly<3>(a.data(), b.data(), P, Ns, j, tw.data()); break;
        default: stockham_bfly<5>(a.data(), b.data(), P, Ns, j, tw.data()); break;
      }
    }
    Ns *= R;
    a.swap(b);
  }
  return a;
}

int main(int argc, char** argv) {
  const long double TWO_PI = 6.283185307179586476925286766559005768L;
  std::mt19937_64 g(1905);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  for (int i = 1; i < argc; ++i) {
    const int P = std::atoi(argv[i]);
    std::vector<double> xr(P), xi(P);
    for (int j = 0; j < P; ++j) {
      xr[j] = u(g);
      xi[j] = u(g);
    }
    std::vector<cd> xd(P), twd(P);
    std::vector<cdw> xw(P), tww(P);
    for (int j = 0; j < P; ++j) {
      xd[j] = cd{xr[j], xi[j]};
      xw[j] = cfrom(xr[j], xi[j], cdw{});
      const long double a = -TWO_PI * j / P;
      twd[j] = cd{(double)cosl(a), (double)sinl(a)};
      tww[j] = cfrom((double)cosl(a), (double)sinl(a), cdw{});
    }
    const std::vector<cd> yd = stockham(xd, P, twd);
    const std::vector<cdw> yw = stockham(xw, P, tww);
    long double ed = 0, ew = 0, nrm = 0;
    for (int k = 0; k < P; ++k) {
      long double sr = 0, si = 0;
      for (int j = 0; j < P; ++j) {
        const long double a = -TWO_PI * (long double)(((long long)j * k) % P) / P;
        sr += xr[j] * cosl(a) - xi[j] * sinl(a);
        si += xr[j] * sinl(a) + xi[j] * cosl(a);
      }
      nrm = fmaxl(nrm, sqrtl(sr * sr + si * si));
      ed = fmaxl(ed, hypotl(yd[k].re - sr, yd[k].im - si));
      ew = fmaxl(ew, hypotl(cre(yw[k]) - sr, cim(yw[k]) - si));
    }
    std::printf("%d %.3Le %.3Le\n", P, ed / nrm, ew / nrm);
  }
  return 0;
}
