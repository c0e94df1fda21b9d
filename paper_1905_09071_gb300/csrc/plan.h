// Device-side description of a plan: what the kernels of one right-hand-side
// evaluation read. Built on the host by the ABI layer, passed by value as a
// __grid_constant__ kernel parameter.
#pragma once

#include <cstdint>

#include "fft_ct.cuh"

namespace sag {

constexpr int kMaxD = 8;
constexpr int kThreads = 256;      // block size of the FFT kernels
constexpr int kRowPosPerThread = 4;  // row kernel: positions owned per thread (2 rows x M2 <= 1024)

// One order d of the system: its FFT geometry and where its data lives.
//
// Complex half-length trick: the real length-L sequence a (index = size,
// a[0] = 0, a[k] = 0 for k > N) is packed as z_j = a[2j] + i a[2j+1],
// j < M = L/2, and z is transformed by a four-step FFT with M = M1 * M2:
// input j = M2 j1 + j2, output k = k1 + M1 k2,
//   Z[k] = sum_{j1} omega_M1^{j1 k1} omega_M^{j2 k1} sum ... (columns j2 first,
//   length M1, then rows k1, length M2).
struct OrderDesc {
  int d, R;            // order and CP rank
  int L, M, M1, M2;    // real FFT length, complex length, four-step factors
  int vbase;           // first global vector index (vectors v = vbase + m R + r)
  int W;               // columns per block in the column kernels
  int ld1, ld2;        // shared-memory leading dimensions (M1 + 1, M2 + 1)
  int ncolblk;         // M2 / W
  int nrowpair;        // floor(M1 / 2) + 1 row pairs {k1, M1 - k1}
  int G;               // vectors per chunk in the row kernel
  int ct1, ct2;        // 1: the column (M1) / row (M2) transforms use the compile-time kernels
  radix_plan rp1, rp2; // radix schedules of M1 and M2
  int64_t scr_off;     // scratch offset (elements) of this order's first vector
  int64_t scr2_off;    // offset of this order's spectral-sum buffer in scratch2
  const void* tw1;     // M1 entries omega_M1^k
  const void* tw2;     // M2 entries omega_M2^k
  const void* tw4;     // M entries omega_M^e (four-step twiddle, e = j2 k1 < M)
  const void* twL;     // M entries omega_L^k, k < M (real-FFT split)
  const float* rscale; // [R] power-of-two weight of rank term r (double-word path)
  double pscale;       // 2^(E_d - d) / (L d!): final scale of P^(d) before the n scale
};

struct DevScalars {
  unsigned long long nmax_bits;  // bits of max |n| (non-negative doubles order like integers)
  int e_n;                       // power-of-two scale of n in the double-word path
  int step;                      // diagnostic row counter of sag_integrate
  double o_stage1;               // outflow at the first stage of an RK2 step
  double cum;                    // cumulative outflow
  double outflow;                // last evaluated outflow
  unsigned int counter;          // last-block detection of the epilogue
  unsigned int status;           // latched device status bits
};

enum : unsigned { kStatusNonFinite = 1u, kStatusTimeout = 2u };

enum EpiMode : int {
  EPI_RHS = 0,       // dndt (and/or p, q parts)
  EPI_HEUN1 = 1,     // k1 = F(n); n* = n + dt k1
  EPI_HEUN2 = 2,     // n <- n + dt/2 (k1 + F(n*))
  EPI_MID1 = 3,      // n* = n + dt/2 F(n)
  EPI_MID2 = 4,      // n <- n + dt F(n*)
};

struct RhsParams {
  int N, D, nord, Vtot, sym, dwpath;
  long long spin_limit;          // clock cycles a bounded device-side wait may take
  int ndotchunk;                 // chunks of the inner-product kernel per vector
  int dotchunk;                  // sizes per chunk
  OrderDesc ord[kMaxD];          // ord[i] describes order d = i + 2
  int colpre[kMaxD + 1];         // prefix sums of column blocks (forward column kernel)
  int rowpre[kMaxD + 1];         // prefix sums of row pairs (row kernel)
  int invpre[kMaxD + 1];         // prefix sums of column blocks (inverse column kernel)
  const double* U64;             // [Vtot][N] FP64 factors
  const float2* Udw;             // [Vtot][N] double-word factors, scaled by 2^-e_v
  float2* ndw;                   // [N] double-word n scaled by 2^-e_n
  void* scratch;                 // forward column output, all vectors
  void* scratch2;                // per order: spectral sum after the inverse row step
  double* pd;                    // [nord][N] P^(d) per order
  double* dot_s;                 // [Vtot][ndotchunk] partial <U, n>
  double* dot_t;                 // [Vtot][ndotchunk] partial <k U, n>
  double* epi_part;              // [gridDim][4] epilogue block partials
  DevScalars* sc;
};

}  // namespace sag
