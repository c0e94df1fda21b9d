// Compile-time Stockham FFT for the transform lengths the plan uses most
// (powers of two and 3 * 2^k from 64 to 768): the radix schedule, spans,
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

SAG_CX bool ct_supported(int P) {
  return P == 64 || P == 128 || P == 256 || P == 512 || P == 96 || P == 192 || P == 384 ||
         P == 768;
}

#if defined(__CUDACC__)
// One in-place pass of radix R and span Ns over COUNT transforms of length P
// (transform b at buf + b * ld), T threads.
template <class C, int P, int R, int Ns, int COUNT, int T>
__device__ __forceinline__ void ct_pass(C* buf, int ld, const C* tw) {
  constexpr int NB = P / R;
  constexpr int TOT = NB * COUNT;
  constexpr int PER = (TOT + T - 1) / T;
  constexpr int TWSTEP = P / (Ns * R);
  C x[PER][R];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int w = threadIdx.x + i * T;
    if (TOT % T == 0 || w < TOT) {
      const int b = w / NB, j = w - b * NB;
      const C* ib = buf + b * ld;
#pragma unroll
      for (int t = 0; t < R; ++t) x[i][t] = ib[j + t * NB];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int w = threadIdx.x + i * T;
    if (TOT % T == 0 || w < TOT) {
      const int b = w / NB, j = w - b * NB;
      const int k = j % Ns;
      if (Ns > 1) {
#pragma unroll
        for (int t = 1; t < R; ++t) x[i][t] = c_mul(x[i][t], tw[t * k * TWSTEP]);
      }
      dft_r<R>(x[i]);
      C* ob = buf + b * ld + (j / Ns) * Ns * R + k;
#pragma unroll
      for (int t = 0; t < R; ++t) ob[t * Ns] = x[i][t];
    }
  }
  __syncthreads();
}

template <class C, int P, int COUNT, int T, int S, int Ns>
__device__ __forceinline__ void ct_passes(C* buf, int ld, const C* tw) {
  constexpr ct_sched sc = make_ct_sched(P);
  if constexpr (S < sc.n) {
    constexpr int R = sc.r[S];
    ct_pass<C, P, R, Ns, COUNT, T>(buf, ld, tw);
    ct_passes<C, P, COUNT, T, S + 1, Ns * R>(buf, ld, tw);
  }
}

// COUNT length-P forward transforms in place; the caller has synchronised
// after filling buf; returns after a barrier with the result in buf.
template <class C, int P, int COUNT, int T>
__device__ __forceinline__ void fft_ct(C* buf, int ld, const C* tw) {
  static_assert(make_ct_sched(P).n > 0, "unsupported compile-time length");
  ct_passes<C, P, COUNT, T, 0, 1>(buf, ld, tw);
}
#endif

}  // namespace sag
