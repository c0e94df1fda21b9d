// Host-side check of the library's FFT building blocks (csrc/dw.cuh, csrc/fft.cuh,
// csrc/fft_ct.cuh): runs the Stockham passes sequentially on the CPU for the
// FP64 and double-word complex types and prints, per length, the max-norm error
// relative to a long-double direct DFT. With "ct" as the first argument it runs
// the compile-time schedule instead, through the same index maps as the device
// passes (padded shared-memory layout, in-place passes, natural-order first
// pass), on several transforms side by side with unused slots set to NaN.
// Compiled by tests/test_fft_host.py with -ffp-contract=off so that float
// operations stay separately rounded.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>

#include "fft.cuh"
#include "fft_ct.cuh"

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

// Compile-time schedule, emulated pass by pass: every butterfly's loads happen
// before any store of the same pass, as in the device code (in place).
template <class C, int P, int S, int Ns>
static void ct_host_passes(std::vector<C>& buf, int ld, int count, const C* tw, const C* nat) {
  constexpr ct_sched sc = make_ct_sched(P);
  if constexpr (S < sc.n) {
    constexpr int R = sc.r[S];
    constexpr int NB = P / R;
    std::vector<C> x((size_t)count * P);
    for (int b = 0; b < count; ++b)
      for (int j = 0; j < NB; ++j)
        for (int t = 0; t < R; ++t) {
          const long src = nat ? (long)b * P + ct_src<P, R, true>(j, t) : (long)b * ld + ct_src<P, R, false>(j, t);
          const long lim = nat ? (long)count * P : (long)count * ld;
          if (src < 0 || src >= lim) {
            std::printf("read out of range P=%d pass %d\n", P, S);
            std::exit(3);
          }
          x[((size_t)b * NB + j) * R + t] = nat ? nat[src] : buf[src];
        }
    for (int b = 0; b < count; ++b)
      for (int j = 0; j < NB; ++j) {
        C* xx = &x[((size_t)b * NB + j) * R];
        std::vector<C> w(R);
        if (Ns > 1)
          for (int t = 1; t < R; ++t) {
            const int ti = ct_twi<P, S, R, Ns>(j, t);
            if (ti < 0 || ti >= ct_twp_size(P) || ct_twp_src(P, ti) < 0) {
              std::printf("twiddle index out of range P=%d pass %d\n", P, S);
              std::exit(3);
            }
            // the global-memory layout names the same twiddle
            const int tg = ct_twg<P, S, R, Ns>(j, t);
            if (tg < 0 || tg >= ct_twg_size(P) || ct_twg_src(P, tg) != ct_twp_src(P, ti)) {
              std::printf("global twiddle table differs P=%d pass %d\n", P, S);
              std::exit(3);
            }
            w[t] = tw[ti];
          }
        // the device passes' butterfly (grid-aligned for double-word radix 2/4/8)
        if (Ns > 1) ct_bfly<R, true>(xx, [&](int t) { return w[t]; });
        else ct_bfly<R, false>(xx, [&](int t) { return w[t]; });
        for (int t = 0; t < R; ++t) {
          const int o = ct_dst<P, R, Ns>(j, t);
          // the last pass's output t of butterfly j is element j + t Ns (natural
          // order), the index the kernels' global-memory last pass stores to
          if (S + 1 == sc.n && o != pad8(j + t * Ns)) {
            std::printf("last pass index differs P=%d\n", P);
            std::exit(3);
          }
          if (o < 0 || o >= ct_span(P) || (long)b * ld + o >= (long)count * ld) {
            std::printf("write out of range P=%d pass %d\n", P, S);
            std::exit(3);
          }
          buf[(size_t)b * ld + o] = xx[t];
        }
      }
    ct_host_passes<C, P, S + 1, Ns * R>(buf, ld, count, tw, nullptr);
  }
}

// count transforms of length P at ld = ct_ld(P, count); sin: the input comes
// from a separate natural-order buffer. Returns the max relative error.
template <int P, class C = cdw>
static long double ct_check(int count, bool sin, std::mt19937_64& g) {
  const long double TWO_PI = 6.283185307179586476925286766559005768L;
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  const int ld = ct_ld(P, count);
  const C nan = cfrom(NAN, NAN, C{});
  std::vector<C> buf((size_t)count * ld, nan), nat((size_t)count * P), tw(P);
  std::vector<double> xr((size_t)count * P), xi((size_t)count * P);
  for (int j = 0; j < P; ++j) {
    const long double a = -TWO_PI * j / P;
    tw[j] = cfrom((double)cosl(a), (double)sinl(a), C{});
  }
  for (int b = 0; b < count; ++b)
    for (int j = 0; j < P; ++j) {
      xr[(size_t)b * P + j] = u(g);
      xi[(size_t)b * P + j] = u(g);
      const C v = cfrom(xr[(size_t)b * P + j], xi[(size_t)b * P + j], C{});
      if (sin) nat[(size_t)b * P + j] = v;
      else buf[(size_t)b * ld + pad8(j)] = v;
    }
  // pass tables, as the kernels build them from the natural table
  std::vector<C> twp(ct_twp_size(P), nan);
  for (int i = 0; i < ct_twp_size(P); ++i)
    if (ct_twp_src(P, i) >= 0) twp[i] = tw[ct_twp_src(P, i)];
  ct_host_passes<C, P, 0, 1>(buf, ld, count, twp.data(), sin ? nat.data() : nullptr);
  long double err = 0, nrm = 0;
  for (int b = 0; b < count; ++b)
    for (int k = 0; k < P; ++k) {
      long double sr = 0, si = 0;
      for (int j = 0; j < P; ++j) {
        const long double a = -TWO_PI * (long double)(((long long)j * k) % P) / P;
        const long double x0 = xr[(size_t)b * P + j], x1 = xi[(size_t)b * P + j];
        sr += x0 * cosl(a) - x1 * sinl(a);
        si += x0 * sinl(a) + x1 * cosl(a);
      }
      const C y = buf[(size_t)b * ld + pad8(k)];
      nrm = fmaxl(nrm, sqrtl(sr * sr + si * si));
      const long double e = hypotl(cre(y) - sr, cim(y) - si);
      if (!(e == e)) return NAN;
      err = fmaxl(err, e);
    }
  return err / nrm;
}

template <class C = cdw>
static long double ct_dispatch(int P, int count, bool sin, std::mt19937_64& g) {
  switch (P) {
    case 64: return ct_check<64, C>(count, sin, g);
    case 96: return ct_check<96, C>(count, sin, g);
    case 128: return ct_check<128, C>(count, sin, g);
    case 192: return ct_check<192, C>(count, sin, g);
    case 256: return ct_check<256, C>(count, sin, g);
    case 384: return ct_check<384, C>(count, sin, g);
    case 512: return ct_check<512, C>(count, sin, g);
    case 768: return ct_check<768, C>(count, sin, g);
    case 1024: return ct_check<1024, C>(count, sin, g);
    case 1536: return ct_check<1536, C>(count, sin, g);
    default: std::printf("unsupported %d\n", P); std::exit(2);
  }
}

int main(int argc, char** argv) {
  const long double TWO_PI = 6.283185307179586476925286766559005768L;
  std::mt19937_64 g(1905);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  if (argc > 1 && std::string(argv[1]) == "ct") {
    // Layouts the kernels use: the column kernels (ct_cols(P) transforms side
    // by side, padded input), the row kernel's chunks (2 ct_group(P)
    // transforms from a natural-order stage) and its inverse (2 transforms).
    for (int i = 2; i < argc; ++i) {
      const int P = std::atoi(argv[i]);
      std::printf("ct %d %d %d %.3Le\n", P, ct_cols(P), 0, ct_dispatch(P, ct_cols(P), false, g));
      // FP64 through the same passes (the plain DFTs of fft.cuh, radix 6 included)
      std::printf("ct64 %d %d %d %.3Le\n", P, ct_cols(P), 0, ct_dispatch<cd>(P, ct_cols(P), false, g));
      if ((P & (P - 1)) == 0 && P <= 512) {
        std::printf("ct %d %d %d %.3Le\n", P, 2 * ct_group(P), 1, ct_dispatch(P, 2 * ct_group(P), true, g));
        std::printf("ct %d %d %d %.3Le\n", P, 2, 0, ct_dispatch(P, 2, false, g));
      }
    }
    return 0;
  }
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
