// Device-side description of a plan: what the kernels of one right-hand-side
// evaluation read. A plan holds B independent systems; each order d of each
// system is one "item" with its own FFT geometry. Item and system tables live
// in device memory; the small RhsParams header is passed by value as a
// __grid_constant__ kernel parameter.
#pragma once

#include <cstdint>

#include "fft_ct.cuh"

namespace sag {

constexpr int kMaxD = 8;
constexpr int kThreads = 256;        // block size of the FFT kernels
constexpr int kRowPosPerThread = 4;  // row kernel: positions owned per thread (2 rows x M2 <= 1024)
constexpr int kMaxTTRank = 16;       // largest TT rank R_lambda the chain kernel holds in registers
constexpr long long kDefaultSpinLimit = 4000000000LL;  // device-side wait limit, cycles (about 2 s)

// One order d of one system: its FFT geometry and where its data lives.
//
// Complex half-length trick: the real length-L sequence a (index = size,
// a[0] = 0, a[k] = 0 for k > N) is packed as z_j = a[2j] + i a[2j+1],
// j < M = L/2, and z is transformed by a four-step FFT with M = M1 * M2:
// input j = M2 j1 + j2, output k = k1 + M1 k2 (columns j2 first, length M1,
// then rows k1, length M2).
struct OrderDesc {
  int sys;             // system index b
  int d, R;            // order and CP rank (TT: unused)
  int nvec;            // factor vectors of this order (CP: d R; TT: nonzero core vectors)
  int N;               // sizes of the system
  int64_t noff;        // offset of the system's size 1 in packed state vectors
  int64_t ndwoff;      // offset of the system's double-word n (RhsParams::ndw)
  int L, M, M1, M2;    // real FFT length, complex length, four-step factors
  int vbase;           // first global vector index (CP: v = vbase + m R + r)
  int W;               // columns per block in the column kernels
  int ld1, ld2;        // shared-memory leading dimensions (M1 + 1, M2 + 1)
  int ncolblk;         // M2 / W
  int nu;              // vectors the forward pass transforms: CP, its distinct vectors
                       // (bitwise); TT, every stored vector (duplicates share one already)
  int umap_off;        // CP with duplicates: offset of its maps in RhsParams::umap/ulist; -1: none
  int nrowpair;        // floor(M1 / 2) + 1 row pairs {k1, M1 - k1}
  int G;               // vectors per chunk in the row kernel
  int ct1, ct2;        // 1: the column (M1) / row (M2) transforms use the compile-time kernels
  int fmt;             // 0 CP, 1 TT
  int ttr[kMaxD + 1];  // TT ranks R_0..R_d (R_0 = R_d = 1)
  int vid_off;         // TT: offset of this order's (lambda, a, b) -> vector table
  radix_plan rp1, rp2; // radix schedules of M1 and M2
  int64_t scr_off;     // scratch offset (elements) of this order's first vector
  int64_t scr2_off;    // offset of this order's spectral-sum buffer in scratch2
  int64_t pd_off;      // offset of P^(d) (N doubles) in the gain buffer
  const void* tw1;     // M1 entries omega_M1^k
  const void* tw2;     // M2 entries omega_M2^k
  const void* tw4;     // M entries omega_M^e (four-step twiddle, e = j2 k1 < M)
  const void* twL;     // M entries omega_L^k, k < M (real-FFT split)
  const void* tw4c;    // compile-time column kernels: omega_M^(j2 k1) in column-block
                       // order (cb, k1, c) with j2 = cb W + c; M entries
  // Pair form of the forward pass (CP, double-word, compile-time kernels, no
  // duplicate vectors): vectors q = 2p, 2p + 1 (rank-major, q = r d + m) are
  // the real and imaginary parts of one length-L sequence, transformed as
  // M1 rows of 2 M2 points; the row pass separates their spectra.
  int pair;            // 1: the forward pass runs on pairs
  int discard;         // pair rows: drop each workspace row's L2 lines once read (128-byte aligned)
  int ctt;             // TT, double-word: the row kernels run compile-time M2-point transforms
  int npair;           // ceil(nvec / 2)
  int ncolblk_p;       // 2 M2 / W column blocks per pair
  int ld2p;            // work-area stride of the pair row transforms
  const void* tw2p;    // pass tables of the 2 M2-point rows, global layout (ct_twg)
  const void* twg2;    // pass tables of the M2-point inverse rows, global layout
  const void* twg1;    // compile-time columns: pass tables of M1, global layout
  const void* tw4c_p;  // omega_L^(j2 k1) for j2 < 2 M2 in column-block order
  int ebase, nent;     // TT: first global core entry, entries (sum_l R_{l-1} R_l)
  int64_t ent_spec_off;// TT: offset (elements) of its entries' cotangent spectra
  int pw;              // 1: the double-word forward columns generate U^(m)_r(i) = u i^a
                       // (RhsParams::vpow, lnt, expk) instead of reading RhsParams::Udw
  const float* rscale; // CP, double-word path: [R] power-of-two weight of rank term r
  double pscale;       // final FP64 scale of P^(d) (1/(L d!), factors of two), before the n scale
  double gscale;       // 2^-d / (L d!): final scale of a vector's cotangent before its exponents
};

// One system of the batch.
struct SysDesc {
  int N, D, fmt;
  int64_t noff;        // packed offset of size 1
  int64_t ndwoff;      // offset of its double-word n (element index = size)
  int vbeg, vend;      // its global vectors
  int dbeg, dend;      // its distinct vectors (the first of each repeated set) in RhsParams::vdist
  int ibeg, iend;      // its items (orders)
  int ndotchunk;       // inner-product chunks per vector
  int epi_beg, epi_blocks;  // its epilogue blocks
};

// Per-system device scalars (one 64-byte line each).
struct SysScalars {
  unsigned long long nmax_bits;  // bits of max |n| (non-negative doubles order like integers)
  unsigned long long gmax_bits;  // bits of max |g| of a vector-Jacobian product's cotangent
  int e_n;                       // power-of-two scale of n in the double-word path
  int e_g;                       // power-of-two scale of the cotangent g
  int step;                      // diagnostic row counter of sag_integrate
  unsigned int counter;          // last-block detection of the epilogue
  double o_stage1;               // outflow at the first stage of an RK2 step
  double cum;                    // cumulative outflow
  double outflow;                // last evaluated outflow
  double gflux;                  // sum_d 1/d! sum_{i in [1,N]^d} |i| C_i prod n (complete first-moment flux)
};

// Latched device status bits. kStatusTimeoutUndrained: a block gave up a
// wait and then also gave up waiting for its own copies in flight.
enum : unsigned { kStatusNonFinite = 1u, kStatusTimeout = 2u, kStatusTimeoutUndrained = 4u };

enum EpiMode : int {
  EPI_RHS = 0,       // dndt (and/or p, q parts)
  EPI_HEUN1 = 1,     // k1 = F(n); n* = n + dt k1
  EPI_HEUN2 = 2,     // n <- n + dt/2 (k1 + F(n*))
  EPI_MID1 = 3,      // n* = n + dt/2 F(n)
  EPI_MID2 = 4,      // n <- n + dt F(n*)
};

struct RhsParams {
  int B, nitems, Vtot, sym, dwpath;
  int exact;                     // double-word path with plain double-word butterflies (cdwx)
  int64_t Ntot;                  // packed state length
  int tt_rmax;                   // largest TT rank of the plan (chain kernel variant)
  int vjp_gmerge;                // CP adjoint rows: g's rows join the vectors' transform batch
  long long spin_limit;          // clock cycles a bounded device-side wait may take
  int wait_unmet;                // test of the timeout path: waits target a barrier nothing completes
  int dotchunk;                  // sizes per inner-product chunk
  int maxdotchunk;               // most chunks of any vector
  const OrderDesc* ord;          // [nitems]
  const SysDesc* sys;            // [B]
  const int* colpre;             // [nitems + 1] forward column kernel blocks (nu per item), in colperm order
  const int* colperm;            // [nitems] items in forward-column table order (by kernel kind in mixed batches)
  const int* colpre_all;         // [nitems + 1] column blocks over every vector (nvec per item; the adjoint)
  const int* umap;               // CP items with duplicates: spectrum slot of vector m R + r (d R entries)
  const int* ulist;              // the same items: vector (m R + r) transformed into slot u (nu entries)
  const int* vrep;               // [Vtot] the first vector bitwise identical to v in v's order (v if unique)
  const int* vdist;              // every system's distinct vectors (vrep[v] == v), SysDesc::dbeg..dend
  const int* rowpre;             // [nitems + 1] row kernel blocks, in rowperm order
  const int* invpre;             // [nitems + 1] inverse column kernel blocks
  const int* chainpre;           // [nitems + 1] TT chain kernel blocks
  const int* epipre;             // [B + 1] epilogue blocks
  const int* vsys;               // [Vtot] system of each vector
  const int* rowperm;            // [nitems] items in row-kernel order, heaviest first (rowpre follows it)
  const double* U64;             // [Vtot][N_b] FP64 factors (vector v at voff[v])
  const int64_t* voff;           // [Vtot] offset of vector v in the factor arrays
  // Double-word copies, indexed by size: element 0 and element N + 1 (and one
  // more for odd N) are zero, elements 1..N hold sizes 1..N, and every array
  // starts on a 16-byte boundary, so that sizes (2j, 2j + 1) form one aligned
  // 16-byte load.
  const float2* Udw;             // factors scaled by 2^-e_v, vector v at vdwoff[v]
  const int64_t* vdwoff;         // [Vtot]
  float2* ndw;                   // n scaled by 2^-e_n of its system, at SysDesc::ndwoff
  // Parametric factors (plans of SAG_CP_POWER systems, double-word path):
  const float4* vpow;            // [Vtot] (u 2^-e_v as hi, lo; a as hi, lo)
  const float2* lnt;             // [max N + 1] ln i as a double-word (entry 0 is 0)
  const float* expk;             // exp constants and table (dw_pow.cuh, kExpConsts floats)
  void* scratch;                 // forward column output, all vectors (TT: then their spectra)
  void* scratch2;                // per item: spectral sum after the inverse row step
  void* spec_nyq;                // TT: [Vtot] Nyquist value of each vector's spectrum
  void* s_nyq;                   // TT: [nitems] Nyquist value of each order's spectral sum
  const int* vid;                // TT: (lambda, a, b) -> vector index or -1, per item
  const float* ewt;              // TT, double-word path: per core entry (parallel to vid) the
                                 // power-of-two weight 2^(e_v - E_lambda) of its vector v in core lambda
  double* pd;                    // gain per item: P^(d) of system b at pd_off
  double* dot_s;                 // [Vtot][maxdotchunk] partial <U, n>
  double* dot_t;                 // [Vtot][maxdotchunk] partial <k U, n>
  double* coef;                  // [Vtot] loss weights: q_k = n_k sum_v coef_v U_v(k)
  double* epi_part;              // [epilogue blocks][4] block partials
  double* qbuf;                  // [Ntot] loss term q of the current evaluation
  // vector-Jacobian product workspace (CP)
  float2* gdw;                   // [Ntot] double-word cotangent scaled by 2^-e_g of its system
  double* gabuf;                 // cotangent of each a = U o n (vector layout, voff)
  double* dot_z;                 // [Vtot][maxdotchunk] partial <U, g o n>
  double* sigma;                 // [Vtot] dL/ds_v through the loss weights
  const int* vexcl;              // [Vtot] sum of the other modes' exponents e_v of the rank term
  // vector-Jacobian product workspace (TT): one cotangent per core entry
  void* ent_spec;                // entries' cotangent spectra, per item at ent_spec_off
  void* ent_nyq;                 // [entries] their Nyquist values
  double* gaent;                 // cotangent of h o n per entry, at eoff
  const int64_t* eoff;           // [entries] offset of an entry's sizes in the core layout
  const int* eexcl;              // [entries] sum of the other cores' exponents E_l of the order
  const int* entpre;             // [nitems + 1] inverse column blocks over the entries
  SysScalars* sc;                // [B]
  unsigned int* status;          // latched device status bits of the plan
};

// Binary search: the largest i in [0, n) with pre[i] <= x (pre[0] = 0, nondecreasing).
__host__ __device__ __forceinline__ int find_segment(const int* pre, int n, int x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

}  // namespace sag
