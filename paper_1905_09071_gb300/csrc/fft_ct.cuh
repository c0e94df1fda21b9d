// Compile-time Stockham FFT for the transform lengths the plan uses most
// (powers of two and 3 * 2^k from 64 to 1536): the radix schedule, spans,
// strides and the thread-to-butterfly map are constants, so index arithmetic
// reduces to shifts and constant multiplies, and each pass works in place in
// one shared-memory buffer (every thread loads all of its butterflies' inputs,
// the block synchronises, then every thread computes and stores), which halves
// the shared memory of the double-buffered generic path.
//
// Schedule: radix 8 while possible, then 4 or 2, then 3: odd radices go last so
// that every span Ns before them is a power of two. The arithmetic of a pass is
// the same Stockham butterfly as the generic path (fft.cuh).
#pragma once

#include <type_traits>

#include "fft.cuh"

#if defined(__CUDACC__)
#define SAG_CX __host__ __device__ constexpr
#else
#define SAG_CX constexpr
#endif

namespace sag {

struct ct_sched {
  int n;
  int r[16];
};

SAG_CX ct_sched make_ct_sched(int P) {
  ct_sched s{0, {0}};
  int odd = 1;
  if (P % 3 == 0) { odd = 3; P /= 3; }
  while (P % 8 == 0) { s.r[s.n++] = 8; P /= 8; }
  if (P == 4) { s.r[s.n++] = 4; P = 1; }
  if (P == 2 && odd == 3) {  // a 2 and the 3 as one radix-6 pass
    s.r[s.n++] = 6;
    return s;
  }
  if (P == 2) { s.r[s.n++] = 2; P = 1; }
  if (odd == 3) s.r[s.n++] = 3;
  if (P != 1) s.n = -1;
  return s;
}

// Columns per block of the compile-time column kernels (about 2048 points per
// block) and vectors per chunk of the compile-time row kernel (about 1024 rows'
// worth of points per transform slot pair).
SAG_CX int ct_cols(int P) {
  int W = 1;
  while (2 * W * P <= 2048) W *= 2;
  return W;
}
SAG_CX int ct_group(int P) { return P >= 1024 ? 1 : 1024 / P; }

// Shared-memory layout of the compile-time kernels. Element i of a transform
// (16-byte complex slots) lives at pad8(i) = i + i / 8: one unused slot after
// every 8, so that the stride-R stores of the first pass and the strided loads
// of the column kernels spread over all eight 16-byte bank groups. A padded
// transform spans ct_span(P) slots; transforms are ct_ld(P, W) slots apart
// when W of them sit side by side (the column kernels fill W columns at
// once). With these, every access of the load, butterfly and store phases is
// free of bank conflicts for the supported lengths (P = 96: 1.08 times the
// conflict-free count).
SAG_CX int pad8(int i) { return i + (i >> 3); }
SAG_CX int ct_span(int P) { return P + P / 8; }
SAG_CX int ct_pad(int W) { return W >= 8 ? 1 : (W == 4 ? 2 : (W == 2 ? 4 : 0)); }
SAG_CX int ct_ld(int P, int W) { return ct_span(P) + ct_pad(W); }

// Padded address of element j + t * STRIDE. When STRIDE is a multiple of 8,
// or j is a multiple of SPAN (> 0) and SPAN divides 8 (the elements of a
// butterfly then share one aligned group of 8), the offset of each t is a
// constant.
template <int STRIDE, int SPAN>
SAG_CX int pad8_at(int j, int t) {
  if constexpr (STRIDE % 8 == 0) return pad8(j) + t * (STRIDE / 8 * 9);
  else if constexpr (SPAN > 0 && 8 % SPAN == 0) return pad8(j) + t * STRIDE;
  else return pad8(j + t * STRIDE);
}

// Butterfly j of a pass of radix R and span Ns over length P: where its t-th
// input is read (natural order if SIN, else padded), where its t-th output is
// written (padded), and the twiddle index of input t.
template <int P, int R, bool SIN>
SAG_CX int ct_src(int j, int t) {
  return SIN ? j + t * (P / R) : pad8_at<P / R, 0>(j, t);
}
template <int P, int R, int Ns>
SAG_CX int ct_dst(int j, int t) {
  return pad8_at<Ns, (Ns == 1 ? R : 0)>((j / Ns) * Ns * R + j % Ns, t);
}

// Twiddles of the compile-time passes, one table per pass s >= 1 (the first
// pass has span 1 and needs none), laid out [k][t - 1] for k = j mod Ns with
// an odd row stride, so that the eight lanes of a 128-bit access phase (eight
// consecutive k) read eight different bank groups. Entry (s, k, t) holds
// omega_P^(t k P / (Ns R)); padding entries (radices with an even R - 1) are
// never read.
SAG_CX int ct_twstride(int R) { return (R - 1) % 2 ? R - 1 : R; }
SAG_CX int ct_twp_off(int P, int S) {
  const ct_sched sc = make_ct_sched(P);
  int off = 0, Ns = sc.r[0];
  for (int s = 1; s < S; ++s) {
    off += Ns * ct_twstride(sc.r[s]);
    Ns *= sc.r[s];
  }
  return off;
}
SAG_CX int ct_twp_size(int P) { return ct_twp_off(P, make_ct_sched(P).n); }
// Index into the natural table (omega_P^e, e < P) of entry i of the pass
// tables, or -1 for a padding entry.
SAG_CX int ct_twp_src(int P, int i) {
  const ct_sched sc = make_ct_sched(P);
  int off = 0, Ns = sc.r[0];
  for (int s = 1; s < sc.n; ++s) {
    const int R = sc.r[s], st = ct_twstride(R);
    if (i < off + Ns * st) {
      const int k = (i - off) / st, t = (i - off) % st + 1;
      return t < R ? t * k * (P / (Ns * R)) : -1;
    }
    off += Ns * st;
    Ns *= R;
  }
  return -1;
}
template <int P, int S, int R, int Ns>
SAG_CX int ct_twi(int j, int t) {
  return ct_twp_off(P, S) + (j % Ns) * ct_twstride(R) + t - 1;
}

// Pass tables in global memory (read through L1, so laid out for coalescing
// rather than for banks): pass s >= 1 holds omega_P^(t k P / (Ns R)) at
// ct_twg_off(P, s) + (t - 1) Ns + k, k < Ns, 1 <= t < R.
SAG_CX int ct_twg_off(int P, int S) {
  const ct_sched sc = make_ct_sched(P);
  int off = 0, Ns = sc.r[0];
  for (int s = 1; s < S; ++s) {
    off += Ns * (sc.r[s] - 1);
    Ns *= sc.r[s];
  }
  return off;
}
SAG_CX int ct_twg_size(int P) { return ct_twg_off(P, make_ct_sched(P).n); }
// Natural-table exponent of entry i of the global pass tables.
SAG_CX int ct_twg_src(int P, int i) {
  const ct_sched sc = make_ct_sched(P);
  int off = 0, Ns = sc.r[0];
  for (int s = 1; s < sc.n; ++s) {
    const int R = sc.r[s];
    if (i < off + Ns * (R - 1)) {
      const int t = (i - off) / Ns + 1, k = (i - off) % Ns;
      return t * k * (P / (Ns * R));
    }
    off += Ns * (R - 1);
    Ns *= R;
  }
  return -1;
}
template <int P, int S, int R, int Ns>
SAG_CX int ct_twg(int j, int t) {
  return ct_twg_off(P, S) + (t - 1) * Ns + j % Ns;
}

// Kernel specialisations (the KIND template argument of k_fwd_col, k_rows and
// k_inv_col): 0 dispatches on the item at run time; 1 is the runtime-length
// path; 2 + i the compile-time length ct_len(i); for k_fwd_col 11 + i the
// pair form at column length ct_len(i); for k_rows 11 + i the pair form at row
// length ct_len(i). The host launches each run of equal kind of the forward
// columns and the rows with its own instantiation, so that a kernel holds one
// path's code and registers (measured: 7% faster than one kernel for every
// path). The inverse columns, about one block per SM, stay one launch.
SAG_CX int ct_len(int i) {
  return i == 0 ? 64 : i == 1 ? 96 : i == 2 ? 128 : i == 3 ? 192 : i == 4 ? 256 : i == 5 ? 384 : i == 6 ? 512
       : i == 7 ? 768 : i == 8 ? 1024 : 1536;
}
constexpr int kCtLengths = 10;
SAG_CX int ct_index(int P) {
  for (int i = 0; i < kCtLengths; ++i)
    if (ct_len(i) == P) return i;
  return -1;
}
constexpr int kKindGeneral = 0, kKindRuntime = 1, kKindCt = 2, kKindPair = kKindCt + kCtLengths,
              kKindCount = kKindPair + kCtLengths;

SAG_CX bool ct_supported(int P) { return ct_index(P) >= 0; }

// The butterfly of a compile-time pass: inputs t >= 1 multiplied by tw(t)
// when TW, then the radix-R DFT. Double-word radix-2/3/4/8 butterflies run in
// the grid-aligned arithmetic of fft_aligned.cuh, the others in dw.cuh's.
template <int R, bool TW, class C, class TWF>
SAG_HD void ct_bfly(C* x, TWF tw) {
  if constexpr (std::is_same<C, cdw>::value && g_radix<R>) {
    g_bfly<R, TW>(x, tw);
  } else {
    if constexpr (TW)
#pragma unroll
      for (int t = 1; t < R; ++t) x[t] = c_mul(x[t], tw(t));
    dft_r<R>(x);
  }
}

#if defined(__CUDACC__)
// Twiddle t of butterfly j: from the shared-memory pass tables (bank layout)
// or, GT, from the global ones (ct_twg layout, read-only path).
template <class C, typename std::enable_if<is_dw<C>::value, int>::type = 0>
__device__ __forceinline__ C ld_ro(const C* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return C(cdw{v.x, v.y, v.z, v.w});
}
__device__ __forceinline__ cd ld_ro(const cd* p) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return cd{v.x, v.y};
}
template <class C, bool GT, int P, int S, int R, int Ns>
__device__ __forceinline__ C tw_at(const C* tw, int j, int t) {
  if constexpr (GT) return ld_ro(tw + ct_twg<P, S, R, Ns>(j, t));
  else return tw[ct_twi<P, S, R, Ns>(j, t)];
}

// One pass of radix R and span Ns over COUNT transforms of length P, T
// threads: transform b is read at src + b * sld (natural order if SIN, else
// padded) and written padded at dst + b * dld. In place (src == dst) the block
// synchronises between the loads and the stores; out of place it does not.
// Ends with a barrier unless TAIL is false.
template <class C, int P, int S, int R, int Ns, int COUNT, int T, bool SIN, bool INPLACE, bool TAIL = true,
          bool GT = false>
__device__ __forceinline__ void ct_pass(const C* src, int sld, C* dst, int dld, const C* tw) {
  constexpr int NB = P / R;
  constexpr int TOT = NB * COUNT;
  constexpr int PER = (TOT + T - 1) / T;
  C x[PER][R];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int w = threadIdx.x + i * T;
    if (TOT % T == 0 || w < TOT) {
      const int b = w / NB, j = w - b * NB;
      const C* ib = src + b * sld;
#pragma unroll
      for (int t = 0; t < R; ++t) x[i][t] = ib[ct_src<P, R, SIN>(j, t)];
    }
  }
  if constexpr (INPLACE) __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int w = threadIdx.x + i * T;
    if (TOT % T == 0 || w < TOT) {
      const int b = w / NB, j = w - b * NB;
      ct_bfly<R, (Ns > 1)>(x[i], [&](int t) { return tw_at<C, GT, P, S, R, Ns>(tw, j, t); });
      C* ob = dst + b * dld;
#pragma unroll
      for (int t = 0; t < R; ++t) ob[ct_dst<P, R, Ns>(j, t)] = x[i][t];
    }
  }
  if constexpr (TAIL) __syncthreads();
}

// Passes S .. END - 1 (END = -1: to the last pass), in place.
template <class C, int P, int COUNT, int T, int S, int Ns, bool GT = false, int END = -1>
__device__ __forceinline__ void ct_passes(C* buf, int ld, const C* tw) {
  constexpr ct_sched sc = make_ct_sched(P);
  constexpr int E = END < 0 ? sc.n : END;
  if constexpr (S < E) {
    constexpr int R = sc.r[S];
    ct_pass<C, P, S, R, Ns, COUNT, T, false, true, true, GT>(buf, ld, buf, ld, tw);
    ct_passes<C, P, COUNT, T, S + 1, Ns * R, GT, END>(buf, ld, tw);
  }
}

// Span (product of the radices before it) of the last pass.
SAG_CX int ct_last_ns(int P) {
  const ct_sched sc = make_ct_sched(P);
  int ns = 1;
  for (int s = 0; s + 1 < sc.n; ++s) ns *= sc.r[s];
  return ns;
}

// First and last passes with their data in global memory, for COUNT
// transforms that sit side by side in the source and destination (the
// columns of a column block). Thread w takes transform b = w mod COUNT and
// butterfly j = w / COUNT, so consecutive threads touch neighbouring columns
// (coalesced global accesses); in the padded layout this map is free of
// bank conflicts as well.
//
// ct_pass_first_from: pass 0 with input element i of transform b from
// load(b, i) (natural order), written padded to dst + b * dld; ends with a
// barrier.
template <class C, int P, int COUNT, int T, class LD>
__device__ __forceinline__ void ct_pass_first_from(LD&& load, C* dst, int dld) {
  constexpr ct_sched sc = make_ct_sched(P);
  constexpr int R = sc.r[0];
  constexpr int NB = P / R;
  constexpr int TOT = NB * COUNT;
  constexpr int PER = (TOT + T - 1) / T;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int w = threadIdx.x + i * T;
    if (TOT % T == 0 || w < TOT) {
      const int b = w % COUNT, j = w / COUNT;
      C x[R];
#pragma unroll
      for (int t = 0; t < R; ++t) x[t] = load(b, j + t * NB);
      ct_bfly<R, false>(x, [&](int) { return C{}; });
      C* ob = dst + b * dld;
#pragma unroll
      for (int t = 0; t < R; ++t) ob[ct_dst<P, R, 1>(j, t)] = x[t];
    }
  }
  __syncthreads();
}

// ct_pass_last_to: the last pass of transforms held padded at src + b * sld
// (after the earlier passes and a barrier), output element k of transform b
// handed to store(b, k, value); no barrier.
template <class C, int P, int COUNT, int T, bool GT, class ST>
__device__ __forceinline__ void ct_pass_last_to(const C* src, int sld, const C* tw, ST&& store) {
  constexpr ct_sched sc = make_ct_sched(P);
  constexpr int S = sc.n - 1;
  constexpr int R = sc.r[S];
  constexpr int Ns = ct_last_ns(P);
  constexpr int NB = P / R;
  constexpr int TOT = NB * COUNT;
  constexpr int PER = (TOT + T - 1) / T;
  static_assert(Ns == NB, "the last pass spans the whole transform");
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int w = threadIdx.x + i * T;
    if (TOT % T == 0 || w < TOT) {
      const int b = w % COUNT, j = w / COUNT;
      const C* ib = src + b * sld;
      C x[R];
#pragma unroll
      for (int t = 0; t < R; ++t) x[t] = ib[ct_src<P, R, false>(j, t)];
      ct_bfly<R, (Ns > 1)>(x, [&](int t) { return tw_at<C, GT, P, S, R, Ns>(tw, j, t); });
#pragma unroll
      for (int t = 0; t < R; ++t) store(b, j + t * Ns, x[t]);
    }
  }
}

// COUNT length-P forward transforms in place in the padded layout; tw holds
// the pass tables (global layout when GT, else the shared-memory layout
// ct_twp_src describes); the caller has synchronised after filling buf;
// returns after a barrier.
template <class C, int P, int COUNT, int T, bool GT = false>
__device__ __forceinline__ void fft_ct(C* buf, int ld, const C* tw) {
  static_assert(make_ct_sched(P).n > 0, "unsupported compile-time length");
  ct_passes<C, P, COUNT, T, 0, 1, GT>(buf, ld, tw);
}

// The same transforms in two steps: fft_ct_first reads natural-order input
// from src (ld sld) and writes the first pass padded to dst, with no barrier
// at the end (src may be refilled once the block has synchronised);
// fft_ct_rest then runs the remaining passes in place in dst, starting after
// the caller's barrier, and returns after a barrier.
template <class C, int P, int COUNT, int T, bool GT = false>
__device__ __forceinline__ void fft_ct_first(const C* src, int sld, C* dst, int dld, const C* tw) {
  static_assert(make_ct_sched(P).n > 1, "unsupported compile-time length");
  constexpr int R = make_ct_sched(P).r[0];
  ct_pass<C, P, 0, R, 1, COUNT, T, true, false, false, GT>(src, sld, dst, dld, tw);
}
template <class C, int P, int COUNT, int T, bool GT = false>
__device__ __forceinline__ void fft_ct_rest(C* buf, int ld, const C* tw) {
  constexpr int R = make_ct_sched(P).r[0];
  ct_passes<C, P, COUNT, T, 1, R, GT>(buf, ld, tw);
}

#endif

}  // namespace sag
