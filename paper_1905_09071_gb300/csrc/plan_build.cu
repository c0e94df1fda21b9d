// Plan construction: validation of the systems, factor vectors (CP modes or
// the nonzero TT core vectors), FFT geometry per (system, order) item,
// twiddle tables, double-word copies with exact power-of-two scaling, block
// tables of every kernel, and the workspace.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "dw_pow.cuh"
#include "plan_host.h"

namespace sag {

// A TT order whose cores hold no nonzero vector (a kernel without that
// order's term) adds nothing to P, and the cotangents of its core entries
// vanish (every product in the chain has a zero factor): it gets no row,
// chain, inverse or entry blocks; its P^(d) and entry cotangents are cleared
// once, when the plan is built.
static bool idle_order(const OrderDesc& od) { return od.fmt == SAG_TT && od.nvec == 0; }
namespace {

double factorial(int d) {
  double f = 1.0;
  for (int i = 2; i <= d; ++i) f *= i;
  return f;
}

// Smallest L = 2^a f with L >= need, f in {1, 3, 5, 15}, or f in {1, 3} only
// (the lengths whose four-step halves have compile-time and pair-form
// kernels in the double-word path: at most 4/3 more points, 2x faster per
// point than the run-time radix kernels a factor 5 would need).
int64_t choose_fft_length(int64_t need, bool allow5 = true) {
  int64_t best = -1;
  const int64_t fs[4] = {1, 3, 5, 15};
  for (int64_t f : fs) {
    if (!allow5 && f % 5 == 0) continue;
    int64_t L = 2 * f;
    while (L < need) L *= 2;
    if (best < 0 || L < best) best = L;
  }
  return best;
}

// omega_P^k = exp(-2 pi i k / P) in FP64.
void unit_root(int64_t k, int64_t P, double& c, double& s) {
  const double a = 2.0 * M_PI * (double)(k % P) / (double)P;
  c = std::cos(a);
  s = -std::sin(a);
}

template <class C>
C to_c(double re, double im);
template <>
cd to_c<cd>(double re, double im) { return cd{re, im}; }
template <>
cdw to_c<cdw>(double re, double im) {
  dw r = dw_from_double(re), i = dw_from_double(im);
  return cdw{r.hi, r.lo, i.hi, i.lo};
}

// Twiddle tables, shared by every item with the same (table length, root order).
template <class C>
struct TwiddleCache {
  std::map<std::pair<int64_t, int64_t>, const void*> tables;
  cudaError_t get(sag_plan_s* pl, int64_t P, int64_t count, const void** out) {
    auto key = std::make_pair(P, count);
    auto it = tables.find(key);
    if (it != tables.end()) {
      *out = it->second;
      return cudaSuccess;
    }
    std::vector<C> h(count);
    for (int64_t k = 0; k < count; ++k) {
      double c, s;
      unit_root(k, P, c, s);
      h[k] = to_c<C>(c, s);
    }
    C* d = nullptr;
    cudaError_t e = pl->upload(&d, h);
    if (e != cudaSuccess) return e;
    tables[key] = d;
    *out = d;
    return cudaSuccess;
  }
  // Pass tables of a compile-time length P in the global layout (ct_twg).
  std::map<int, const void*> pass_tables;
  cudaError_t get_pass(sag_plan_s* pl, int P, const void** out) {
    auto it = pass_tables.find(P);
    if (it != pass_tables.end()) {
      *out = it->second;
      return cudaSuccess;
    }
    std::vector<C> h(std::max(1, ct_twg_size(P)));
    for (int i = 0; i < ct_twg_size(P); ++i) {
      double c, s;
      unit_root(ct_twg_src(P, i), P, c, s);
      h[i] = to_c<C>(c, s);
    }
    C* d = nullptr;
    cudaError_t e = pl->upload(&d, h);
    if (e != cudaSuccess) return e;
    pass_tables[P] = d;
    *out = d;
    return cudaSuccess;
  }
  // omega_M^(j2 k1) for M = M1 M2 in the order the compile-time column kernel
  // reads it: column block cb (W columns), then k1, then column c, j2 = cb W + c.
  std::map<std::tuple<int, int, int>, const void*> col_tables;
  cudaError_t get_col(sag_plan_s* pl, int M1, int M2, int W, const void** out) {
    auto key = std::make_tuple(M1, M2, W);
    auto it = col_tables.find(key);
    if (it != col_tables.end()) {
      *out = it->second;
      return cudaSuccess;
    }
    const int64_t M = (int64_t)M1 * M2;
    std::vector<C> h(M);
    int64_t i = 0;
    for (int cb = 0; cb < M2 / W; ++cb)
      for (int k1 = 0; k1 < M1; ++k1)
        for (int c = 0; c < W; ++c) {
          double cs, sn;
          unit_root((int64_t)(cb * W + c) * k1, M, cs, sn);
          h[i++] = to_c<C>(cs, sn);
        }
    C* d = nullptr;
    cudaError_t e = pl->upload(&d, h);
    if (e != cudaSuccess) return e;
    col_tables[key] = d;
    *out = d;
    return cudaSuccess;
  }
};

template <class C>
cudaError_t item_tables(sag_plan_s* pl, TwiddleCache<C>& tc, OrderDesc& od) {
  cudaError_t e = tc.get(pl, od.M1, od.M1, &od.tw1);
  if (e == cudaSuccess) e = tc.get(pl, od.M2, od.M2, &od.tw2);
  if (e == cudaSuccess) e = tc.get(pl, od.M, od.M, &od.tw4);
  if (e == cudaSuccess) e = tc.get(pl, od.L, od.M, &od.twL);
  od.tw4c = nullptr;
  if (e == cudaSuccess && od.ct1) e = tc.get_col(pl, od.M1, od.M2, od.W, &od.tw4c);
  od.tw2p = nullptr;
  od.twg2 = nullptr;
  od.twg1 = nullptr;
  od.tw4c_p = nullptr;
  if (e == cudaSuccess && od.ct1) e = tc.get_pass(pl, od.M1, &od.twg1);
  if (e == cudaSuccess && od.pair) e = tc.get_pass(pl, 2 * od.M2, &od.tw2p);
  if (e == cudaSuccess && (od.ct2 || od.ctt)) e = tc.get_pass(pl, od.M2, &od.twg2);
  if (e == cudaSuccess && od.pair) e = tc.get_col(pl, od.M1, 2 * od.M2, od.W, &od.tw4c_p);
  return e;
}

int64_t factor_count(const sag_system& s) {
  int64_t nf = 0;
  const int32_t* rk = s.rank;
  for (int d = 2; d <= s.D; ++d) {
    if (s.fmt == SAG_CP) {
      nf += (int64_t)d * rk[0] * s.N;
      rk += 1;
    } else {
      for (int l = 1; l <= d; ++l) nf += (int64_t)rk[l - 1] * rk[l] * s.N;
      rk += d + 1;
    }
  }
  return nf;
}

}  // namespace

sag_status validate_systems(const sag_system* sys, int32_t B, const sag_options& opt) {
  if (!sys) return fail(SAG_EINVAL, "sys is NULL");
  if (B < 1) return fail(SAG_EINVAL, "B must be >= 1");
  if (B > 65535) return fail(SAG_EINVAL, "B must be <= 65535");
  if (opt.prec != SAG_FP64 && opt.prec != SAG_FP32_SPLIT && opt.prec != SAG_FP32_SPLIT_EXACT)
    return fail(SAG_EINVAL, "unknown precision");
  if (opt.rk != SAG_HEUN && opt.rk != SAG_MIDPOINT) return fail(SAG_EINVAL, "unknown RK2 variant");
  if (opt.symmetrize_q != 0 && opt.symmetrize_q != 1) return fail(SAG_EINVAL, "symmetrize_q must be 0 or 1");
  if (opt.autotune != 0 && opt.autotune != 1) return fail(SAG_EINVAL, "autotune must be 0 or 1");
  if (opt.keep_repeats != 0 && opt.keep_repeats != 1) return fail(SAG_EINVAL, "keep_repeats must be 0 or 1");
  if (opt.max_m2 != 0 && (opt.max_m2 < 4 || opt.max_m2 > 512 || (opt.max_m2 & (opt.max_m2 - 1)) != 0))
    return fail(SAG_EINVAL, "max_m2 must be 0 or a power of two in [4, 512]");
  if ((opt.m2 == nullptr) != (opt.n_m2 == 0) || opt.n_m2 < 0)
    return fail(SAG_EINVAL, "m2 and n_m2 go together (NULL and 0, or n_m2 >= 1 values)");
  for (int i = 0; i < opt.n_m2; ++i) {
    const int u = opt.m2[i];
    if (u != 0 && (u < 4 || u > 512 || (u & (u - 1)) != 0))
      return fail(SAG_EINVAL, "m2 entries must be 0 or powers of two in [4, 512]");
  }
  for (int b = 0; b < B; ++b) {
    const sag_system& s = sys[b];
    const std::string at = B > 1 ? " (system " + std::to_string(b) + ")" : "";
    if (s.N < 1) return fail(SAG_EINVAL, "N must be >= 1" + at);
    if (s.N > (1 << 22)) return fail(SAG_EUNSUPPORTED, "N above 2^22" + at);
    if (s.D < 2 || s.D > kMaxD) return fail(SAG_EINVAL, "D must be in [2, 8]" + at);
    if (!s.rank) return fail(SAG_EINVAL, "rank is NULL" + at);
    if (!s.factors) return fail(SAG_EINVAL, "factors is NULL" + at);
    if (s.fmt != SAG_CP && s.fmt != SAG_TT) return fail(SAG_EINVAL, "unknown format" + at);
    if (s.fmt != sys[0].fmt) return fail(SAG_EUNSUPPORTED, "all systems of a plan must share one format" + at);
    const int32_t* rk = s.rank;
    int present = 0;
    for (int d = 2; d <= s.D; ++d) {
      if (s.fmt == SAG_CP) {
        if (rk[0] < 0 || rk[0] > 4096) return fail(SAG_EINVAL, "CP rank out of [0, 4096]" + at);
        present += rk[0] > 0;
        rk += 1;
      } else {
        if (rk[0] != 1 || rk[d] != 1) return fail(SAG_EINVAL, "TT ranks must start and end with 1" + at);
        for (int l = 1; l < d; ++l)
          if (rk[l] < 1 || rk[l] > kMaxTTRank) return fail(SAG_EINVAL, "TT rank out of [1, 16]" + at);
        present += 1;
        rk += d + 1;
      }
    }
    if (present == 0) return fail(SAG_EINVAL, "every CP rank is 0: the system has no kernel" + at);
    if (factor_count(s) > ((int64_t)1 << 34)) return fail(SAG_EINVAL, "factor array too large" + at);
  }
  return SAG_OK;
}

sag_status build_plan(const sag_system* sys, int32_t B, const sag_options& opt, sag_plan_s* pl) {
  const bool dwp = opt.prec == SAG_FP32_SPLIT || opt.prec == SAG_FP32_SPLIT_EXACT;
  const bool tt = sys[0].fmt == SAG_TT;
  const size_t csize = dwp ? sizeof(cdw) : sizeof(cd);
  pl->B = B;
  pl->prec = opt.prec;
  pl->rk = opt.rk;
  pl->sym = opt.symmetrize_q;
  pl->fmt = sys[0].fmt;
  RhsParams& P = pl->P;
  P.B = B;
  P.sym = opt.symmetrize_q;
  P.dwpath = dwp ? 1 : 0;
  P.exact = opt.prec == SAG_FP32_SPLIT_EXACT ? 1 : 0;
  P.spin_limit = kDefaultSpinLimit;
  P.dotchunk = 8192;

  // ---- vectors: host copy of every nonzero factor vector, packed ----------
  std::vector<double> hf;          // concatenated vectors
  std::vector<int64_t> voff;       // offset of each vector in hf
  std::vector<int64_t> vdwoff;     // offset of each vector in the double-word copy
  std::vector<int> vsys;           // system of each vector
  std::vector<int> vid;            // TT tables
  std::vector<int> umap, ulist;    // CP duplicate maps
  std::vector<SysDesc>& S = pl->systems;
  std::vector<OrderDesc>& I = pl->items;
  S.resize(B);
  pl->offsets.assign(B + 1, 0);
  int64_t noff = 0, ndwoff = 0, vdwtot = 0;
  // Double-word arrays are indexed by size with zero slots at 0 and N + 1
  // (one more for odd N, so that every array starts 16-byte aligned).
  auto dwlen = [](int N) { return (int64_t)((N + 3) & ~1); };
  cudaError_t e;
  for (int b = 0; b < B; ++b) {
    const sag_system& s = sys[b];
    const int N = s.N;
    const int64_t nf = factor_count(s);
    std::vector<double> src((size_t)nf);
    e = cudaMemcpy(src.data(), s.factors, (size_t)nf * sizeof(double),
                   s.factors_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
    if (e != cudaSuccess) return cuda_fail(e, "copy factors");
    for (double x : src)
      if (!std::isfinite(x)) return fail(SAG_EINVAL, "factors contain Inf or NaN");
    SysDesc& sd = S[b];
    sd.N = N;
    sd.D = s.D;
    sd.fmt = s.fmt;
    sd.noff = noff;
    sd.ndwoff = ndwoff;
    sd.vbeg = (int)vsys.size();
    sd.ibeg = (int)I.size();
    sd.ndotchunk = (N + P.dotchunk - 1) / P.dotchunk;
    const int32_t* rk = s.rank;
    int64_t soff = 0;  // offset in the caller's factor array
    for (int d = 2; d <= s.D; ++d) {
      if (s.fmt == SAG_CP && rk[0] == 0) {  // rank 0: the order is absent
        rk += 1;
        continue;
      }
      OrderDesc od{};
      od.sys = b;
      od.d = d;
      od.N = N;
      od.noff = noff;
      od.ndwoff = ndwoff;
      od.fmt = s.fmt;
      od.vbase = (int)vsys.size();
      auto push_vector = [&](const double* x) {
        voff.push_back((int64_t)hf.size());
        vdwoff.push_back(vdwtot);
        vdwtot += dwlen(N);
        vsys.push_back(b);
        hf.insert(hf.end(), x, x + N);
        return (int)vsys.size() - 1;
      };
      if (s.fmt == SAG_CP) {
        od.R = rk[0];
        od.nvec = d * od.R;
        for (int v = 0; v < od.nvec; ++v) push_vector(src.data() + soff + (int64_t)v * N);
        // Bitwise-identical vectors of the order are transformed once: slot
        // umap[v] holds the spectrum of vector ulist[umap[v]].
        std::vector<int> um(od.nvec), ul;
        std::map<uint64_t, std::vector<int>> seen;
        for (int v = 0; v < od.nvec; ++v) {
          const double* x = src.data() + soff + (int64_t)v * N;
          uint64_t h = 1469598103934665603ull;  // FNV-1a over the bytes
          const unsigned char* bytes = reinterpret_cast<const unsigned char*>(x);
          for (size_t k = 0; k < (size_t)N * sizeof(double); ++k) h = (h ^ bytes[k]) * 1099511628211ull;
          int found = -1;
          if (!opt.keep_repeats)  // else every vector is its own slot (its factors may change)
            for (int u : seen[h])
              if (std::memcmp(x, src.data() + soff + (int64_t)ul[u] * N, (size_t)N * sizeof(double)) == 0) {
                found = u;
                break;
              }
          if (found < 0) {
            found = (int)ul.size();
            ul.push_back(v);
            seen[h].push_back(found);
          }
          um[v] = found;
        }
        od.nu = (int)ul.size();
        od.umap_off = -1;
        if (od.nu < od.nvec) {
          od.umap_off = (int)umap.size();
          umap.insert(umap.end(), um.begin(), um.end());
          ulist.insert(ulist.end(), ul.begin(), ul.end());
          ulist.resize(umap.size(), 0);  // both tables indexed from umap_off
        }
        soff += (int64_t)od.nvec * N;
        rk += 1;
      } else {
        od.R = 0;
        for (int l = 0; l <= d; ++l) od.ttr[l] = rk[l];
        od.vid_off = (int)vid.size();
        int cnt = 0;
        // Bitwise-identical vectors of the order's cores share one id, hence one
        // transform (the Theorem-1 cores repeat the same powers in every core);
        // the power-of-two weight, which depends on the core, is per entry.
        std::vector<std::pair<const double*, int>> core;
        for (int l = 1; l <= d; ++l) {
          for (int a = 0; a < rk[l - 1]; ++a)
            for (int c = 0; c < rk[l]; ++c) {
              const double* x = src.data() + soff;
              soff += N;
              bool nz = false;
              for (int k = 0; k < N && !nz; ++k) nz = x[k] != 0.0;
              int id = -1;
              if (nz) {
                for (const auto& pc : core)
                  if (std::memcmp(x, pc.first, (size_t)N * sizeof(double)) == 0) id = pc.second;
                if (id < 0) {
                  id = push_vector(x);
                  core.push_back({x, id});
                  ++cnt;
                }
              }
              vid.push_back(id);
            }
        }
        od.nvec = cnt;
        od.nu = cnt;
        od.umap_off = -1;
        rk += d + 1;
        for (int l = 0; l <= d; ++l) P.tt_rmax = std::max(P.tt_rmax, od.ttr[l]);
      }
      I.push_back(od);
    }
    sd.vend = (int)vsys.size();
    sd.iend = (int)I.size();
    noff += N;
    ndwoff += dwlen(N);
    pl->offsets[b + 1] = noff;
  }
  pl->Ntot = noff;
  pl->nfactor = (int64_t)hf.size();
  pl->nfactor_dw = vdwtot;
  P.Ntot = noff;
  P.Vtot = (int)vsys.size();
  P.nitems = (int)I.size();
  const int Vtot = P.Vtot;
  if (Vtot == 0) return fail(SAG_EINVAL, "every kernel is identically zero");
  // Repeated vectors (the slot maps of CP orders): the loss term's inner
  // products and factor passes use one vector of each repeated set.
  std::vector<int> vrep(Vtot), vdist;
  for (int v = 0; v < Vtot; ++v) vrep[v] = v;
  for (const OrderDesc& od : I)
    if (od.fmt == SAG_CP && od.umap_off >= 0)
      for (int q = 0; q < od.nvec; ++q) vrep[od.vbase + q] = od.vbase + ulist[od.umap_off + umap[od.umap_off + q]];
  for (SysDesc& sd : S) {
    sd.dbeg = (int)vdist.size();
    for (int v = sd.vbeg; v < sd.vend; ++v)
      if (vrep[v] == v) vdist.push_back(v);
    sd.dend = (int)vdist.size();
  }

  // ---- FFT geometry of each item ------------------------------------------
  if (opt.m2 && opt.n_m2 != (int)I.size())
    return fail(SAG_EINVAL, "m2 needs one entry per order of the plan (" + std::to_string(I.size()) + ")");
  int64_t scr = 0, scr2 = 0, pdo = 0;
  size_t col_smem = 0, row_smem = 0, rowtt_smem = 0;
  size_t vrow_merged = 0;  // adjoint row blocks with g's rows in the vectors' batch
  std::vector<size_t> item_col_smem, item_row_smem;  // per item: what its column / row blocks need
  std::vector<int> colpre(1, 0), colpre_all(1, 0), invpre(1, 0), chainpre(1, 0);
  std::vector<int> entpre(1, 0);  // TT adjoint: inverse column blocks over the core entries
  int nent_tot = 0;
  int64_t entspec = 0;
  for (OrderDesc& od : I) {
    const int d = od.d;
    const int64_t L = choose_fft_length(std::max<int64_t>((int64_t)d * od.N, 16), !dwp);
    if (L > (int64_t)1 << 24) return fail(SAG_EUNSUPPORTED, "FFT length above 2^24 (d N too large)");
    od.L = (int)L;
    od.M = (int)(L / 2);
    // Four-step split M = M1 M2: M2 by the rule (capped by max_m2), or the
    // geometry autotuner's choice for this item.
    const int m2cap = opt.max_m2 > 0 ? opt.max_m2 : 512;
    int M2 = 1;
    while ((int64_t)(2 * M2) * (2 * M2) <= od.M && 2 * M2 <= m2cap && od.M % (2 * M2) == 0) M2 *= 2;
    const size_t ix = (size_t)(&od - I.data());
    if (opt.m2 && opt.m2[ix] > 0) {
      if (od.M % opt.m2[ix] != 0 || od.M / opt.m2[ix] > 4096)
        return fail(SAG_EINVAL, "m2 entry " + std::to_string(ix) + " must divide M = " + std::to_string(od.M) +
                                    " with M / M2 <= 4096");
      M2 = opt.m2[ix];
    }
    if (ix < pl->m2_pref.size() && pl->m2_pref[ix] > 0 && od.M % pl->m2_pref[ix] == 0) M2 = pl->m2_pref[ix];
    od.M2 = M2;
    od.M1 = od.M / M2;
    if (od.M1 > 4096) return fail(SAG_EUNSUPPORTED, "FFT column length above 4096");
    od.rp1 = make_radix_plan(od.M1);
    od.rp2 = make_radix_plan(od.M2);
    if (od.rp1.n < 0 || od.rp2.n < 0) return fail(SAG_EUNSUPPORTED, "FFT length not a supported product");
    // Compile-time kernels (double-word path) for the common lengths; the
    // compile-time row kernel serves CP only.
    od.ct1 = (dwp && ct_supported(od.M1) && M2 >= ct_cols(od.M1)) ? 1 : 0;
    od.ct2 = (dwp && !tt && ct_supported(od.M2) && od.M2 <= 512) ? 1 : 0;
    od.ctt = (dwp && tt && (od.M2 == 64 || od.M2 == 128 || od.M2 == 256 || od.M2 == 512)) ? 1 : 0;
    int W = 1;
    while (2 * W <= M2 && (int64_t)2 * W * od.M1 <= 2048) W *= 2;
    if (od.ct1) W = ct_cols(od.M1);
    od.W = W;
    // The compile-time column kernels pad their transforms per column count.
    od.ld1 = od.ct1 ? ct_ld(od.M1, W) : od.M1 + 1;
    od.ncolblk = M2 / W;
    od.nrowpair = od.M1 / 2 + 1;
    int G = std::max(1, 2048 / (2 * M2));
    G = std::min(G, std::max(1, od.nvec));
    G = std::min(G, 64);
    if (od.ct2) G = ct_group(od.M2);
    od.ld2 = od.ct2 ? ct_ld(od.M2, 2 * G) : od.M2 + 1;
    if (dwp && !tt && !od.ct2 && 2 * od.M2 > kThreads)
      return fail(SAG_EUNSUPPORTED, "row length without a compile-time kernel above 128");
    od.G = G;
    // Pairs (see OrderDesc): rows of 2 M2 points with a compile-time kernel,
    // columns of at most 1024 points (the pair column kernels' lengths; the
    // rule never pairs 1536-point columns, whose rows are 2 x 512 points).
    od.pair = 0;
    od.discard = 0;
    od.npair = 0;
    od.ncolblk_p = 0;
    od.ld2p = 0;
    if (od.ct1 && od.ct2 && !tt && od.umap_off < 0 && od.M1 <= 1024 && 2 * od.M2 <= 512 &&
        ct_supported(2 * od.M2)) {
      od.pair = 1;
      od.npair = (od.nvec + 1) / 2;
      od.ncolblk_p = 2 * M2 / W;
      od.ld2p = ct_ld(2 * od.M2, 2 * ct_group(2 * od.M2));
    }
    od.scr_off = scr;
    scr += (int64_t)std::max(od.nvec, 2 * od.npair) * od.M;
    // The pair rows drop their workspace lines from L2 once read: every row
    // (2 M2 points, at pair p row k1: scr_off + 2 M p + 2 M2 k1 elements of
    // 16 bytes) must start on a 128-byte line of the 256-byte aligned buffer.
    if (od.pair && dwp && od.scr_off % 8 == 0 && (2 * od.M) % 8 == 0 && (2 * od.M2) % 8 == 0) od.discard = 1;
    od.scr2_off = scr2;
    scr2 += od.M;
    od.pd_off = pdo;
    pdo += od.N;
    colpre.push_back(colpre.back() + (od.pair ? od.npair * od.ncolblk_p : od.nu * od.ncolblk));
    colpre_all.push_back(colpre_all.back() + od.nvec * od.ncolblk);
    invpre.push_back(invpre.back() + (idle_order(od) ? 0 : od.ncolblk));
    chainpre.push_back(chainpre.back() + (tt && !idle_order(od) ? (od.M + 1 + 255) / 256 : 0));
    od.nent = 0;
    if (tt)
      for (int l = 1; l <= d; ++l) od.nent += od.ttr[l - 1] * od.ttr[l];
    od.ebase = nent_tot;
    nent_tot += od.nent;
    od.ent_spec_off = entspec;
    entspec += (int64_t)od.nent * od.M;
    entpre.push_back(entpre.back() + (idle_order(od) ? 0 : od.nent * od.ncolblk));
    // Compile-time kernels work in place (one buffer, pass tables in global
    // memory), the generic ones ping-pong and keep the natural table.
    item_col_smem.push_back(od.ct1 ? (size_t)(W * od.ld1) * csize : (size_t)(2 * W * od.ld1 + od.M1) * csize);
    col_smem = std::max(col_smem, item_col_smem.back());
    // The compile-time row kernels stage their input (bulk copies, natural
    // order) apart from the padded work area, behind one mbarrier: 2 G
    // transforms of M2 points, or in the pair form 2 G' transforms of 2 M2
    // points. The runtime one ping-pongs.
    if (od.pair) {
      const int Gp = ct_group(2 * od.M2);
      item_row_smem.push_back((size_t)(2 * Gp * 2 * od.M2 + 2 * Gp * od.ld2p) * csize + 16);
    } else {
      item_row_smem.push_back(od.ct2 ? (size_t)(2 * G * od.M2 + 2 * G * od.ld2) * csize + 16
                                     : (size_t)(2 * G * 2 * od.ld2 + od.M2) * csize);
    }
    row_smem = std::max(row_smem, item_row_smem.back());
    rowtt_smem = std::max(rowtt_smem, (size_t)std::max(2 * G * 2 * od.ld2, 6 * od.ld2) * csize +
                                          (size_t)od.M2 * csize);
    if (od.ctt)  // compile-time TT rows: 2 ct_group(M2) padded slots forward; sums and 2 slots inverse
      rowtt_smem = std::max(rowtt_smem, (size_t)std::max(2 * ct_group(od.M2) * ct_ld(od.M2, 2 * ct_group(od.M2)),
                                                          2 * od.M2 + 2 * ct_ld(od.M2, 2)) * csize);
    // Vector-Jacobian product kernels (CP): ping-pong column blocks; row
    // blocks hold the d vectors of a rank term, g's spectrum and d spectra.
    pl->L.vcol_smem = std::max(pl->L.vcol_smem, (size_t)(2 * W * od.ld1 + od.M1) * csize);
    pl->L.vrow_smem = std::max(pl->L.vrow_smem, (size_t)(4 * d * od.ld2 + (d + 1) * (2 * od.M2 + 1) +
                                                         od.M2) * csize);
    vrow_merged = std::max(vrow_merged, (size_t)(4 * (d + 1) * od.ld2 + (d + 1) * (2 * od.M2 + 1) +
                                                 od.M2) * csize);  // g's rows in the vectors' batch
  }
  // Row blocks: items with the most vectors first.
  std::vector<int> rowperm(I.size());
  for (size_t i = 0; i < I.size(); ++i) rowperm[i] = (int)i;
  std::stable_sort(rowperm.begin(), rowperm.end(),
                   [&](int a, int b) { return I[a].nvec > I[b].nvec; });
  std::vector<int> rowpre(1, 0);
  for (int i : rowperm) rowpre.push_back(rowpre.back() + (idle_order(I[i]) ? 0 : I[i].nrowpair));
  // Epilogue blocks per system; largest vector count per system.
  std::vector<int> epipre(1, 0);
  int maxnv = 1, maxchunk = 1;
  for (SysDesc& sd : S) {
    sd.epi_beg = epipre.back();
    sd.epi_blocks = (sd.N + 255) / 256;
    epipre.push_back(epipre.back() + sd.epi_blocks);
    maxnv = std::max(maxnv, sd.vend - sd.vbeg);
    maxchunk = std::max(maxchunk, sd.ndotchunk);
  }
  P.maxdotchunk = maxchunk;

  LaunchCfg& L = pl->L;
  int maxN = 1;
  for (const SysDesc& sd : S) maxN = std::max(maxN, sd.N);
  // n's max and split: a grid of (blocks, B) with a grid-stride loop; about
  // four blocks per SM in all, at least 64 per system
  int nsm = 152;
  {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      nsm = v;
  }
  L.prep_blocks = std::max(1, std::min((maxN + 255) / 256, std::max(64, (4 * nsm + B - 1) / B)));
  L.col_blocks = colpre.back();
  L.col_blocks_all = colpre_all.back();
  L.row_blocks = rowpre.back();
  L.inv_blocks = invpre.back();
  L.chain_blocks = chainpre.back();
  // The adjoint rows transform g with the vectors when d + 1 slots fit.
  P.vjp_gmerge = (!tt && vrow_merged > 0 && (int)vrow_merged <= smem_limit()) ? 1 : 0;
  if (P.vjp_gmerge) L.vrow_smem = vrow_merged;
  L.vjp_rmax = 1;
  for (const OrderDesc& od : I) L.vjp_rmax = std::max(L.vjp_rmax, od.R);
  L.ent_blocks = entpre.back();
  L.epi_blocks = epipre.back();
  L.has_tt = tt ? 1 : 0;
  L.col_smem = col_smem;
  L.row_smem = row_smem;
  L.inv_smem = col_smem;
  // Each launch of one kernel specialisation gets the shared memory its own
  // items need (the largest item of another kind would cut the occupancy of
  // every launch); the run-time dispatching kernel keeps the plan's largest.
  for (int k = 0; k < kKindCount; ++k) L.col_smem_kind[k] = L.row_smem_kind[k] = 0;
  for (size_t i = 0; i < I.size(); ++i) {
    const OrderDesc& od = I[i];
    if (!dwp) break;
    const int ck = od.ct1 ? kKindCt + ct_index(od.M1) : kKindRuntime;
    L.col_smem_kind[ck] = std::max(L.col_smem_kind[ck], item_col_smem[i]);  // single vectors (adjoint too)
    if (od.pair) {
      const int pk = kKindPair + ct_index(od.M1);
      L.col_smem_kind[pk] = std::max(L.col_smem_kind[pk], item_col_smem[i]);
    }
    if (!tt) {
      const int rk = od.pair ? kKindPair + ct_index(2 * od.M2) : od.ct2 ? kKindCt + ct_index(od.M2) : kKindRuntime;
      L.row_smem_kind[rk] = std::max(L.row_smem_kind[rk], item_row_smem[i]);
    }
  }
  L.col_smem_kind[kKindGeneral] = col_smem;
  L.row_smem_kind[kKindGeneral] = row_smem;
  L.rowtt_smem = rowtt_smem;
  L.epi_smem = (size_t)2 * maxnv * sizeof(double);  // k_qterm: weights, and the folded ones of repeats
  L.coef_smem = (size_t)2 * maxnv * sizeof(double);
  if (col_smem > 227 * 1024 || row_smem > 227 * 1024 || rowtt_smem > 227 * 1024 ||
      L.coef_smem > 200 * 1024)
    return fail(SAG_EUNSUPPORTED, "shared-memory footprint above the per-block limit (too many vectors)");

  // ---- factor copies --------------------------------------------------------
  double* U64 = nullptr;
  if ((e = pl->upload(&U64, hf)) != cudaSuccess) return fail(SAG_ENOMEM, "cudaMalloc factors");
  P.U64 = U64;
  // Double-word copy: each vector scaled by 2^-e_v so that max |U| lies in
  // [0.5, 1). CP: rank term r of an order carries 2^(sigma_r - E) with
  // sigma_r = sum_m e_{v(m,r)}, E = max_r sigma_r. TT: vector v of core l
  // carries 2^(e_v - E_l), E_l = max over the core. The remaining 2^E (CP) or
  // 2^(sum_l E_l) (TT) moves into the FP64 scale of P^(d).
  std::vector<int> ev(Vtot, 0);
  if (dwp) {
    std::vector<float2> hdw((size_t)std::max<int64_t>(vdwtot, 1), make_float2(0.f, 0.f));
    for (int v = 0; v < Vtot; ++v) {
      const int N = S[vsys[v]].N;
      const double* x = hf.data() + voff[v];
      double mx = 0.0;
      for (int k = 0; k < N; ++k) mx = std::max(mx, std::fabs(x[k]));
      int ex = 0;
      if (mx > 0.0) std::frexp(mx, &ex);
      ev[v] = ex;
      for (int k = 0; k < N; ++k) {
        dw y = dw_from_double(std::ldexp(x[k], -ex));
        hdw[vdwoff[v] + 1 + k] = make_float2(y.hi, y.lo);
      }
    }
    float2* Udw = nullptr;
    if ((e = pl->upload(&Udw, hdw)) != cudaSuccess) return fail(SAG_ENOMEM, "cudaMalloc dw factors");
    P.Udw = Udw;
    if (!pl->pow_ua.empty() && !P.exact) {
      // Parametric factors (SAG_FP32_SPLIT; the exact double-word path reads
      // the stored copy): per vector (u 2^-e_v, a) as double-words, ln i per
      // size (the largest N of the plan), and the exp constants.
      if ((int64_t)pl->pow_ua.size() != 2 * (int64_t)Vtot) return fail(SAG_EINVAL, "power parameters do not match the vectors");
      std::vector<float4> vp(Vtot);
      for (int v = 0; v < Vtot; ++v) {
        const dw u = dw_from_double(std::ldexp(pl->pow_ua[2 * v], -ev[v]));
        const dw a = dw_from_double(pl->pow_ua[2 * v + 1]);
        vp[v] = make_float4(u.hi, u.lo, a.hi, a.lo);
      }
      int nmax = 1;
      for (const SysDesc& sd : S) nmax = std::max(nmax, sd.N);
      std::vector<float2> lt((size_t)nmax + 1, make_float2(0.f, 0.f));
      for (int i = 1; i <= nmax; ++i) {
        const long double l = logl((long double)i);
        const float hi = (float)l;
        lt[i] = make_float2(hi, (float)(l - hi));
      }
      std::vector<float> ek(kExpConsts);
      make_exp_consts(ek.data());
      float4* dvp = nullptr;
      float2* dlt = nullptr;
      float* dek = nullptr;
      if ((e = pl->upload(&dvp, vp)) != cudaSuccess || (e = pl->upload(&dlt, lt)) != cudaSuccess ||
          (e = pl->upload(&dek, ek)) != cudaSuccess)
        return fail(SAG_ENOMEM, "cudaMalloc power tables");
      P.vpow = dvp;
      P.lnt = dlt;
      P.expk = dek;
      for (OrderDesc& od : I) od.pw = 1;
    }
    float2* ndw = nullptr;
    if ((e = pl->alloc(&ndw, (size_t)std::max<int64_t>(ndwoff, 1))) != cudaSuccess)
      return fail(SAG_ENOMEM, "cudaMalloc n");
    // the zero slots stay zero: the split kernel writes elements 1..N only
    if ((e = cudaMemset(ndw, 0, (size_t)std::max<int64_t>(ndwoff, 1) * sizeof(float2))) != cudaSuccess)
      return cuda_fail(e, "clear n");
    P.ndw = ndw;
  }
  std::vector<float> ewt(std::max<size_t>(vid.size(), 1), 1.0f);
  std::vector<int> eexcl((size_t)std::max(nent_tot, 1), 0);  // TT: the other cores' exponents per entry
  TwiddleCache<cdw> tcw;
  TwiddleCache<cd> tcd;
  for (OrderDesc& od : I) {
    const int d = od.d;
    int Esum = 0;
    if (dwp && od.fmt == SAG_CP) {
      std::vector<int> sig(od.R, 0);
      for (int r = 0; r < od.R; ++r)
        for (int m = 0; m < d; ++m) sig[r] += ev[od.vbase + m * od.R + r];
      Esum = *std::max_element(sig.begin(), sig.end());
      std::vector<float> rs(od.R);
      for (int r = 0; r < od.R; ++r) rs[r] = std::ldexp(1.0f, sig[r] - Esum);
      float* drs = nullptr;
      if ((e = pl->upload(&drs, rs)) != cudaSuccess) return fail(SAG_ENOMEM, "cudaMalloc rank scales");
      od.rscale = drs;
    } else if (dwp) {
      int off = od.vid_off;
      std::vector<int> Els(d + 1, 0);
      for (int l = 1; l <= d; ++l) {
        const int cnt = od.ttr[l - 1] * od.ttr[l];
        int El = INT32_MIN;
        for (int j = 0; j < cnt; ++j)
          if (vid[off + j] >= 0) El = std::max(El, ev[vid[off + j]]);
        if (El == INT32_MIN) El = 0;
        for (int j = 0; j < cnt; ++j)
          if (vid[off + j] >= 0) ewt[off + j] = std::ldexp(1.0f, ev[vid[off + j]] - El);
        Els[l] = El;
        Esum += El;
        off += cnt;
      }
      int eo = od.ebase;
      for (int l = 1; l <= d; ++l)
        for (int j = 0; j < od.ttr[l - 1] * od.ttr[l]; ++j) eexcl[eo++] = Esum - Els[l];
    }
    e = dwp ? item_tables<cdw>(pl, tcw, od) : item_tables<cd>(pl, tcd, od);
    if (e != cudaSuccess) return cuda_fail(e, "twiddle tables");
    // A factor 2 per mode comes from the real split (2 A[k]), 1/L from the
    // unnormalised inverse, 1/d! from the definition of p^(d).
    od.pscale = std::ldexp(1.0, Esum - d) / ((double)od.L * factorial(d));
    od.gscale = std::ldexp(1.0, -d) / ((double)od.L * factorial(d));
  }
  // Vector-Jacobian product: exponent sum of the other modes of each CP vector.
  std::vector<int> vexcl(Vtot, 0);
  if (!tt)
    for (const OrderDesc& od : I)
      for (int m = 0; m < od.d; ++m)
        for (int r = 0; r < od.R; ++r) {
          int sum = 0;
          for (int mm = 0; mm < od.d; ++mm)
            if (mm != m) sum += ev[od.vbase + mm * od.R + r];
          vexcl[od.vbase + m * od.R + r] = sum;
        }

  // ---- workspace and tables ---------------------------------------------------
  void* scratch = nullptr;
  void* scratch2 = nullptr;
  if ((e = pl->alloc((unsigned char**)&scratch, (size_t)std::max<int64_t>(scr, 1) * csize)) != cudaSuccess ||
      (e = pl->alloc((unsigned char**)&scratch2, (size_t)scr2 * csize)) != cudaSuccess)
    return fail(SAG_ENOMEM, "cudaMalloc FFT workspace");
  P.scratch = scratch;
  P.scratch2 = scratch2;
  OrderDesc* d_ord = nullptr;
  SysDesc* d_sys = nullptr;
  // Forward-column table order: the items' natural order, or the items sorted
  // by kernel specialisation when that order alternates between more kinds
  // than the launcher issues launches for (mixed batches); the table then
  // holds one run per kind. colpre follows this order.
  std::vector<int> colkind_nat(I.size()), colperm(I.size());
  for (size_t i = 0; i < I.size(); ++i) {
    const OrderDesc& od = I[i];
    const int ct = od.ct1 ? kKindCt + ct_index(od.M1) : kKindRuntime;
    colkind_nat[i] = !dwp ? kKindGeneral : od.pair ? kKindPair + ct_index(od.M1) : ct;
  }
  pl->col_sorted = kind_order(colkind_nat.data(), (int)I.size(), colperm.data());
  std::vector<int> colpre_t(1, 0), colkind_t;
  for (int i : colperm) {
    colpre_t.push_back(colpre_t.back() + colpre[i + 1] - colpre[i]);
    colkind_t.push_back(colkind_nat[i]);
  }
  int *d_colpre = nullptr, *d_colpre_all = nullptr, *d_umap = nullptr, *d_ulist = nullptr, *d_colperm = nullptr,
      *d_rowpre = nullptr, *d_invpre = nullptr, *d_chainpre = nullptr,
      *d_epipre = nullptr, *d_vsys = nullptr, *d_rowperm = nullptr, *d_vid = nullptr;
  int64_t* d_voff = nullptr;
  int64_t* d_vdwoff = nullptr;
  float* d_vw = nullptr;
  int* d_vrep = nullptr;
  int* d_vdist = nullptr;
  if (pl->upload(&d_ord, I) != cudaSuccess || pl->upload(&d_sys, S) != cudaSuccess ||
      pl->upload(&d_colpre, colpre_t) != cudaSuccess || pl->upload(&d_colperm, colperm) != cudaSuccess ||
      pl->upload(&d_rowpre, rowpre) != cudaSuccess ||
      pl->upload(&d_colpre_all, colpre_all) != cudaSuccess || pl->upload(&d_umap, umap) != cudaSuccess ||
      pl->upload(&d_ulist, ulist) != cudaSuccess ||
      pl->upload(&d_invpre, invpre) != cudaSuccess || pl->upload(&d_chainpre, chainpre) != cudaSuccess ||
      pl->upload(&d_epipre, epipre) != cudaSuccess || pl->upload(&d_vsys, vsys) != cudaSuccess ||
      pl->upload(&d_rowperm, rowperm) != cudaSuccess || pl->upload(&d_vid, vid) != cudaSuccess ||
      pl->upload(&d_voff, voff) != cudaSuccess || pl->upload(&d_vw, ewt) != cudaSuccess ||
      pl->upload(&d_vdwoff, vdwoff) != cudaSuccess || pl->upload(&d_vrep, vrep) != cudaSuccess ||
      pl->upload(&d_vdist, vdist) != cudaSuccess)
    return fail(SAG_ENOMEM, "cudaMalloc tables");
  P.vrep = d_vrep;
  P.vdist = d_vdist;
  pl->h_umap = umap;  // for the checks of sag_plan_update_factors
  pl->h_ulist = ulist;
  P.ord = d_ord;
  P.sys = d_sys;
  P.colpre = d_colpre;
  P.colperm = d_colperm;
  P.colpre_all = d_colpre_all;
  P.umap = d_umap;
  P.ulist = d_ulist;
  P.rowpre = d_rowpre;
  P.invpre = d_invpre;
  P.chainpre = d_chainpre;
  P.epipre = d_epipre;
  P.vsys = d_vsys;
  P.rowperm = d_rowperm;
  P.vid = d_vid;
  P.voff = d_voff;
  P.vdwoff = d_vdwoff;
  P.ewt = d_vw;
  const size_t Nt = (size_t)pl->Ntot;
  if (pl->alloc((unsigned char**)&P.spec_nyq, (size_t)Vtot * csize) != cudaSuccess ||
      pl->alloc((unsigned char**)&P.s_nyq, (size_t)P.nitems * csize) != cudaSuccess ||
      pl->alloc(&P.pd, (size_t)pdo) != cudaSuccess ||
      pl->alloc(&P.dot_s, (size_t)Vtot * P.maxdotchunk) != cudaSuccess ||
      pl->alloc(&P.dot_t, (size_t)Vtot * P.maxdotchunk) != cudaSuccess ||
      pl->alloc(&P.coef, (size_t)std::max(Vtot, nent_tot)) != cudaSuccess ||
      pl->alloc(&pl->epi_part, (size_t)L.epi_blocks * 4) != cudaSuccess ||
      pl->alloc(&P.sc, (size_t)B) != cudaSuccess || pl->alloc(&P.status, 1) != cudaSuccess ||
      pl->alloc(&pl->nstar, Nt) != cudaSuccess || pl->alloc(&pl->k1buf, Nt) != cudaSuccess ||
      pl->alloc(&pl->stage_a, Nt) != cudaSuccess || pl->alloc(&pl->stage_b, Nt) != cudaSuccess ||
      pl->alloc(&pl->stage_c, Nt) != cudaSuccess || pl->alloc(&pl->dev_outflow, (size_t)B) != cudaSuccess ||
      pl->alloc(&P.qbuf, Nt) != cudaSuccess)
    return fail(SAG_ENOMEM, "cudaMalloc workspace");
  P.epi_part = pl->epi_part;
  if (!tt) {
    int* d_vexcl = nullptr;
    if (pl->upload(&d_vexcl, vexcl) != cudaSuccess || pl->alloc(&P.gabuf, hf.size()) != cudaSuccess ||
        pl->alloc(&P.dot_z, (size_t)Vtot * P.maxdotchunk) != cudaSuccess ||
        pl->alloc(&P.sigma, (size_t)Vtot) != cudaSuccess ||
        (dwp && pl->alloc(&P.gdw, Nt) != cudaSuccess))
      return fail(SAG_ENOMEM, "cudaMalloc adjoint workspace");
    P.vexcl = d_vexcl;
  } else {
    // TT adjoint: one cotangent per core entry, in the caller's core layout
    // (eoff), so entries without a stored vector get theirs too.
    std::vector<int64_t> eoff((size_t)std::max(nent_tot, 1), 0);
    int64_t cur = 0;
    for (const OrderDesc& od : I)
      for (int q = 0; q < od.nent; ++q) {
        eoff[od.ebase + q] = cur;
        cur += od.N;
      }
    pl->nfactor = cur;
    int *d_eexcl = nullptr, *d_entpre = nullptr;
    int64_t* d_eoff = nullptr;
    if (pl->upload(&d_eexcl, eexcl) != cudaSuccess || pl->upload(&d_entpre, entpre) != cudaSuccess ||
        pl->upload(&d_eoff, eoff) != cudaSuccess ||
        pl->alloc((unsigned char**)&P.ent_spec, (size_t)std::max<int64_t>(entspec, 1) * csize) != cudaSuccess ||
        pl->alloc((unsigned char**)&P.ent_nyq, (size_t)std::max(nent_tot, 1) * csize) != cudaSuccess ||
        pl->alloc(&P.gaent, (size_t)std::max<int64_t>(cur, 1)) != cudaSuccess ||
        pl->alloc(&P.dot_z, (size_t)Vtot * P.maxdotchunk) != cudaSuccess ||
        pl->alloc(&P.sigma, (size_t)std::max(nent_tot, 1)) != cudaSuccess ||
        (dwp && pl->alloc(&P.gdw, Nt) != cudaSuccess))
      return fail(SAG_ENOMEM, "cudaMalloc adjoint workspace");
    P.eexcl = d_eexcl;
    P.entpre = d_entpre;
    P.eoff = d_eoff;
    // entries of idle orders keep zero cotangents (no kernel writes them)
    if ((e = cudaMemset(P.gaent, 0, sizeof(double) * (size_t)std::max<int64_t>(cur, 1))) != cudaSuccess)
      return cuda_fail(e, "memset");
  }
  if ((e = cudaMemset(P.sc, 0, sizeof(SysScalars) * B)) != cudaSuccess ||
      (e = cudaMemset(P.status, 0, sizeof(unsigned))) != cudaSuccess ||
      (e = cudaMemset(P.pd, 0, sizeof(double) * (size_t)std::max<int64_t>(pdo, 1))) != cudaSuccess)  // idle orders' P^(d)
    return cuda_fail(e, "memset");

  e = setup_common_kernels(L);
  if (e == cudaSuccess) e = dwp ? setup_fft_kernels_dw(L) : setup_fft_kernels_f64(L);
  if (e == cudaSuccess) e = setup_vjp_common(L);
  if (e == cudaSuccess && !dwp) e = setup_vjp_fft_f64(L);  // the dw paths' are in setup_fft_kernels_dw
  if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
  if ((e = cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&pl->side.stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&pl->side.fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&pl->side.join, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "stream");
  // Stream groups of the FFT stage. Default: in the double-word path, a plan
  // with 2 to 4 CP items (one system) runs one FFT chain per item on its own
  // stream (the FP64 kernels, bound by the FP64 pipe, gain nothing from the
  // overlap and lose a little); else one launch per kernel. With autotune the
  // plan times 1..4 groups instead.
  pl->h_colpre = colpre_t;
  pl->h_colpre_all = colpre_all;
  pl->h_invpre = invpre;
  // Kernel specialisation of the column table entries (table order; the row
  // table's follow its order, set by configure_fft_groups). The adjoint's
  // table over every vector keeps the item order.
  pl->h_colkind = colkind_t;
  pl->h_colkind_all.resize(I.size());
  for (size_t i = 0; i < I.size(); ++i) {
    const OrderDesc& od = I[i];
    pl->h_colkind_all[i] = dwp ? (od.ct1 ? kKindCt + ct_index(od.M1) : kKindRuntime) : kKindGeneral;
  }
  const int ni = (int)I.size();
  pl->L.col = KindTable{pl->h_colpre.data(), pl->h_colkind.data(), ni};
  pl->L.col_all = KindTable{pl->h_colpre_all.data(), pl->h_colkind_all.data(), ni};
  pl->h_nrowpair.resize(I.size());
  pl->h_nvec.resize(I.size());
  pl->h_work.resize(I.size());
  for (size_t i = 0; i < I.size(); ++i) {
    pl->h_nrowpair[i] = idle_order(I[i]) ? 0 : I[i].nrowpair;
    pl->h_nvec[i] = I[i].nvec;
    pl->h_work[i] = (double)I[i].nvec * (double)I[i].M;
  }
  sag_status st = configure_fft_groups(pl, (!tt && dwp && P.nitems <= kMaxFftGroups) ? P.nitems : 1);
  if (st == SAG_OK && opt.autotune && !tt && P.nitems >= 2) st = autotune_fft_groups(pl);
  if (st != SAG_OK) return st;
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "plan setup");
  return SAG_OK;
}

// Splits the items into G groups of consecutive items (balanced by FFT
// points; G = number of items: one item each), orders the row blocks group by
// group (heaviest group first, heaviest items first within it), uploads that
// order and sets the groups' block ranges and streams (heaviest group at the
// highest priority). G = 1: one launch per kernel over every item.
sag_status configure_fft_groups(sag_plan_s* pl, int G) {
  RhsParams& P = pl->P;
  const int n = P.nitems;
  G = std::max(1, std::min(G, std::min(n, (int)kMaxFftGroups)));
  if (pl->col_sorted) G = 1;  // groups take consecutive items of the item-ordered tables
  std::vector<int> cut(G + 1, 0);
  cut[G] = n;
  if (G == n) {
    for (int g = 0; g <= G; ++g) cut[g] = g;
  } else if (G > 1) {
    double total = 0.0;
    for (double w : pl->h_work) total += w;
    double acc = 0.0;
    int g = 1;
    for (int i = 0; i < n && g < G; ++i) {
      acc += pl->h_work[i];
      // cut after item i once its share is reached, leaving an item for each later group
      if (acc >= total * g / G && n - (i + 1) >= G - g) cut[g++] = i + 1;
    }
    for (; g < G; ++g) cut[g] = n - (G - g);  // (only when the shares were not reached)
  }
  std::vector<int> chunk(G);
  std::vector<double> cw(G, 0.0);
  for (int g = 0; g < G; ++g) {
    chunk[g] = g;
    for (int i = cut[g]; i < cut[g + 1]; ++i) cw[g] += pl->h_work[i];
  }
  std::stable_sort(chunk.begin(), chunk.end(), [&](int a, int b) { return cw[a] > cw[b]; });
  std::vector<int> rowperm, rowpre(1, 0), rstart(G + 1, 0);
  for (int c = 0; c < G; ++c) {
    const int g = chunk[c];
    std::vector<int> items;
    for (int i = cut[g]; i < cut[g + 1]; ++i) items.push_back(i);
    std::stable_sort(items.begin(), items.end(), [&](int a, int b) { return pl->h_nvec[a] > pl->h_nvec[b]; });
    for (int i : items) {
      rowperm.push_back(i);
      rowpre.push_back(rowpre.back() + pl->h_nrowpair[i]);
    }
    rstart[c + 1] = (int)rowperm.size();
  }
  // Row kernel specialisation of each item (kKindGeneral for TT plans, whose
  // rows run other kernels, and for FP64).
  auto row_kind = [&](int item) {
    const OrderDesc& od = pl->items[item];
    if (!P.dwpath || pl->fmt == SAG_TT) return (int)kKindGeneral;
    return od.pair ? kKindPair + ct_index(2 * od.M2) : od.ct2 ? kKindCt + ct_index(od.M2) : kKindRuntime;
  };
  if (G == 1) {
    // one launch per kind: order the rows by kind where the heaviest-first
    // order alternates between more kinds than launches (heaviest first
    // within each kind)
    std::vector<int> kinds(n), ord(n);
    for (int j = 0; j < n; ++j) kinds[j] = row_kind(rowperm[j]);
    if (kind_order(kinds.data(), n, ord.data())) {
      std::vector<int> rp(n);
      for (int j = 0; j < n; ++j) rp[j] = rowperm[ord[j]];
      rowperm = rp;
      for (int j = 0; j < n; ++j) rowpre[j + 1] = rowpre[j] + pl->h_nrowpair[rowperm[j]];
    }
  }
  cudaError_t e;
  if ((e = cudaMemcpy((void*)P.rowperm, rowperm.data(), sizeof(int) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy((void*)P.rowpre, rowpre.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice)) !=
          cudaSuccess)
    return cuda_fail(e, "row block order");
  // Row kernel specialisation per row-table entry.
  pl->h_rowperm = rowperm;
  pl->h_rowpre = rowpre;
  pl->h_rowkind.resize(n);
  for (int j = 0; j < n; ++j) pl->h_rowkind[j] = row_kind(rowperm[j]);
  pl->L.row = KindTable{pl->h_rowpre.data(), pl->h_rowkind.data(), n};
  pl->groups.n = 0;
  pl->fft_groups = G;
  if (G == 1) return SAG_OK;
  int least = 0, greatest = 0;
  if ((e = cudaDeviceGetStreamPriorityRange(&least, &greatest)) != cudaSuccess) return cuda_fail(e, "stream");
  for (int c = 0; c < G; ++c) {
    const int g = chunk[c];
    const int i0 = cut[g], i1 = cut[g + 1];
    pl->groups.r[c] = FftRange{pl->h_colpre[i0], pl->h_colpre[i1], rowpre[rstart[c]], rowpre[rstart[c + 1]],
                               pl->h_invpre[i0], pl->h_invpre[i1]};
    SideStream& s = pl->groups.s[c];
    if (!s.stream) {
      const int prio = std::min(least, greatest + c);
      if ((e = cudaStreamCreateWithPriority(&s.stream, cudaStreamNonBlocking, prio)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&s.join, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "stream");
      s.fork = nullptr;
    }
  }
  pl->groups.n = G;
  return SAG_OK;
}

namespace {

// Mean time of one RK2 step (the two stages that sag_integrate replays, with
// dt = 0 so that the state in the staging buffer does not change), replayed
// as a graph with the plan's current groups.
sag_status time_step_graph(sag_plan_s* pl, float* ms) {
  EpiArgs a{};
  a.mode = pl->rk == SAG_HEUN ? EPI_HEUN1 : EPI_MID1;
  a.nin = pl->stage_a;
  a.out0 = pl->nstar;
  a.k1buf = pl->k1buf;
  a.part = pl->epi_part;
  a.split_next = pl->P.dwpath;  // as enqueue_step does
  EpiArgs b{};
  b.mode = pl->rk == SAG_HEUN ? EPI_HEUN2 : EPI_MID2;
  b.nin = pl->nstar;
  b.nbase = pl->stage_a;
  b.k1buf = pl->k1buf;
  b.part = pl->epi_part;
  b.presplit = pl->P.dwpath;
  cudaStream_t cs = pl->cap_stream;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "autotune capture");
  cudaError_t el = enqueue_eval(pl->P, pl->L, pl->stage_a, a, cs, nullptr, &pl->side, &pl->groups);
  if (el == cudaSuccess) el = enqueue_eval(pl->P, pl->L, pl->nstar, b, cs, nullptr, &pl->side, &pl->groups);
  e = cudaStreamEndCapture(cs, &g);
  if (el != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(el != cudaSuccess ? el : e, "autotune capture");
  }
  e = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "autotune instantiate");
  if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaGraphLaunch(x, cs);
    if (e == cudaSuccess) e = cudaEventRecord(e0, cs);
    for (int i = 0; i < 10 && e == cudaSuccess; ++i) e = cudaGraphLaunch(x, cs);
    if (e == cudaSuccess) e = cudaEventRecord(e1, cs);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGraphExecDestroy(x);
  if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
  *ms /= 10.0f;
  return SAG_OK;
}

}  // namespace

namespace {

// The autotuners' input: n = e^{-k/10} per system, normalised to M0 = 1, in
// the plan's input staging buffer.
sag_status load_tuning_input(sag_plan_s* pl) {
  std::vector<double> h((size_t)pl->Ntot);
  for (const SysDesc& sd : pl->systems) {
    double s = 0.0;
    for (int k = 1; k <= sd.N; ++k) s += std::exp(-k / 10.0);
    for (int k = 1; k <= sd.N; ++k) h[sd.noff + k - 1] = std::exp(-k / 10.0) / s;
  }
  cudaError_t e = cudaMemcpy(pl->stage_a, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? SAG_OK : cuda_fail(e, "autotune input");
}

}  // namespace

// Times 1..4 stream groups on this plan (synthetic n = e^{-k/10} per system),
// three sweeps over the candidates, each candidate's best time counting, and
// keeps the fewest groups within 1% of the fastest.
sag_status autotune_fft_groups(sag_plan_s* pl) {
  sag_status st = load_tuning_input(pl);
  if (st != SAG_OK) return st;
  const int gmax = pl->col_sorted ? 1 : std::min(pl->P.nitems, (int)kMaxFftGroups);
  float t[kMaxFftGroups + 1];
  for (int G = 1; G <= gmax; ++G) t[G] = 1e30f;
  for (int sweep = 0; sweep < 3; ++sweep)
    for (int G = 1; G <= gmax; ++G) {
      sag_status s = configure_fft_groups(pl, G);
      float ms = 0.0f;
      if (s == SAG_OK) s = time_step_graph(pl, &ms);
      if (s != SAG_OK) return s;
      t[G] = std::min(t[G], ms);
    }
  float fastest = t[1];
  for (int G = 2; G <= gmax; ++G) fastest = std::min(fastest, t[G]);
  int best_g = 1;
  while (t[best_g] > 1.01f * fastest) ++best_g;
  return configure_fft_groups(pl, best_g);
}

namespace {

// An alternative four-step split M = M1 M2 for the pair form: both the
// column length M1 (at most 1024) and the pair rows' 2 M2 points have
// compile-time kernels, and a column block's W columns fit in M2 columns.
bool pair_split_ok(int M, int M2) {
  if (M2 < 4 || M % (2 * M2) != 0) return false;
  const int M1 = M / M2;
  return ct_supported(M1) && M1 <= 1024 && ct_supported(M2) && ct_supported(2 * M2) && 2 * M2 <= 512 &&
         M2 >= ct_cols(M1);
}

// Best of three timings of one graph-replayed RK2 step on the tuning input.
sag_status time_plan(sag_plan_s* pl, float* ms) {
  sag_status st = load_tuning_input(pl);
  *ms = 1e30f;
  for (int rep = 0; rep < 3 && st == SAG_OK; ++rep) {
    float t = 0.0f;
    st = time_step_graph(pl, &t);
    *ms = std::min(*ms, t);
  }
  return st;
}

// Appends one candidate (its splits [M1, M2] per order, time, verdict) to log.
void log_geometry(std::string& log, const sag_plan_s* of, float ms, bool kept) {
  std::string js = "{\"splits\": [";
  for (size_t i = 0; i < of->items.size(); ++i)
    js += std::string(i ? ", " : "") + "[" + std::to_string(of->items[i].M1) + ", " +
          std::to_string(of->items[i].M2) + "]";
  char t[32];
  std::snprintf(t, sizeof t, "%.4f", ms);
  js += std::string("], \"ms_per_step\": ") + t + ", \"kept\": " + (kept ? "true" : "false") + "}";
  log += (log.empty() ? "" : ", ") + js;
}

}  // namespace

// Coordinate search over the four-step split of each order of a double-word
// CP plan with 1 to 4 orders (the pair form): for each order in turn, a
// whole plan is built with that order's M2 halved (where both lengths still
// have compile-time kernels, so that the candidate keeps the pair form) and
// timed as graph-replayed RK2 steps against the best plan so far; a candidate
// replaces it when it is more than 1% faster. The kept plan's describe()
// lists every candidate with its time.
sag_status autotune_geometry(const sag_system* sys, int32_t B, const sag_options& opt, sag_plan_s** plp) {
  sag_plan_s* best = *plp;
  const int n = (int)best->items.size();
  if (opt.m2 || !best->P.dwpath || best->fmt != SAG_CP || n > kMaxFftGroups) return SAG_OK;
  std::vector<int> pref(n);
  bool any = false;
  for (int i = 0; i < n; ++i) {
    const OrderDesc& od = best->items[i];
    pref[i] = od.M2;
    any = any || (od.pair && pair_split_ok(od.M, od.M2 / 2));
  }
  if (!any) return SAG_OK;
  float best_ms = 0.0f;
  sag_status st = time_plan(best, &best_ms);
  if (st != SAG_OK) return st;
  std::string log;
  log_geometry(log, best, best_ms, true);
  for (int i = 0; i < n; ++i) {
    const OrderDesc& od = best->items[i];
    const int alt = od.M2 / 2;
    if (!od.pair || !pair_split_ok(od.M, alt)) continue;
    sag_plan_s* cand = new (std::nothrow) sag_plan_s();
    if (!cand) return fail(SAG_ENOMEM, "host allocation");
    cand->m2_pref = pref;
    cand->m2_pref[i] = alt;
    cand->pow_ua = best->pow_ua;
    float ms = 0.0f;
    st = build_plan(sys, B, opt, cand);
    // A candidate that cannot be built (device memory) or that lost the
    // pair form is skipped; the plan so far stays valid.
    if (st != SAG_OK || !cand->items[i].pair || cand->items[i].M2 != alt) {
      cudaDeviceSynchronize();
      delete cand;
      continue;
    }
    st = time_plan(cand, &ms);
    if (st != SAG_OK) {
      cudaDeviceSynchronize();
      delete cand;
      return st;
    }
    const bool keep = ms < 0.99f * best_ms;
    log_geometry(log, cand, ms, keep);
    cudaDeviceSynchronize();
    if (keep) {
      delete best;
      best = cand;
      *plp = best;  // the caller owns the plan kept so far
      best_ms = ms;
      pref[i] = alt;
    } else {
      delete cand;
    }
  }
  best->tune_log = log;
  return SAG_OK;
}

}  // namespace sag

namespace sag {

// New values for the factors of a CP plan (same systems, ranks and layout):
// the FP64 and double-word copies, the power-of-two scales and the tables
// that depend on them are rewritten in place; nothing is allocated, so
// captured graphs stay valid.
sag_status update_factors(sag_plan_s* pl, const double* factors, int on_device) {
  if (pl->fmt != SAG_CP) return fail(SAG_EUNSUPPORTED, "factor updates need a CP plan");
  if (!pl->pow_ua.empty())
    return fail(SAG_EUNSUPPORTED, "a plan of parametric factors (SAG_CP_POWER) takes no factor updates");
  RhsParams& P = pl->P;
  const bool dwp = P.dwpath != 0;
  const int Vtot = P.Vtot;
  const size_t nf = (size_t)pl->nfactor;
  std::vector<double> hf(nf);
  cudaError_t e = cudaMemcpy(hf.data(), factors, nf * sizeof(double),
                             on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
  if (e != cudaSuccess) return cuda_fail(e, "copy factors");
  for (double x : hf)
    if (!std::isfinite(x)) return fail(SAG_EINVAL, "factors contain Inf or NaN");
  {
    // Vectors that share a transform (bitwise identical at plan time) must
    // stay identical: the forward pass transforms only the first of them.
    std::vector<int64_t> vo(Vtot);
    if ((e = cudaMemcpy(vo.data(), P.voff, sizeof(int64_t) * Vtot, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "read layout");
    for (const OrderDesc& od : pl->items) {
      if (od.umap_off < 0) continue;
      for (int q = 0; q < od.nvec; ++q) {
        const int rep = pl->h_ulist[od.umap_off + pl->h_umap[od.umap_off + q]];
        if (rep != q && std::memcmp(hf.data() + vo[od.vbase + q], hf.data() + vo[od.vbase + rep],
                                    (size_t)od.N * sizeof(double)) != 0)
          return fail(SAG_EINVAL, "the new factors make vectors differ that were identical when the plan was "
                                  "made (they share one transform); build the plan with keep_repeats = 1");
      }
    }
  }
  if ((e = cudaMemcpy((void*)P.U64, hf.data(), nf * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "upload factors");
  std::vector<int> ev(Vtot, 0);
  std::vector<int64_t> voff(Vtot), vdwoff(Vtot);
  if ((e = cudaMemcpy(voff.data(), P.voff, sizeof(int64_t) * Vtot, cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(vdwoff.data(), P.vdwoff, sizeof(int64_t) * Vtot, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "read layout");
  if (dwp) {
    std::vector<float2> hdw((size_t)pl->nfactor_dw, make_float2(0.f, 0.f));
    for (const SysDesc& sd : pl->systems)
      for (int v = sd.vbeg; v < sd.vend; ++v) {
        const double* x = hf.data() + voff[v];
        double mx = 0.0;
        for (int k = 0; k < sd.N; ++k) mx = std::max(mx, std::fabs(x[k]));
        int ex = 0;
        if (mx > 0.0) std::frexp(mx, &ex);
        ev[v] = ex;
        for (int k = 0; k < sd.N; ++k) {
          dw y = dw_from_double(std::ldexp(x[k], -ex));
          hdw[vdwoff[v] + 1 + k] = make_float2(y.hi, y.lo);
        }
      }
    if ((e = cudaMemcpy((void*)P.Udw, hdw.data(), hdw.size() * sizeof(float2), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return cuda_fail(e, "upload dw factors");
  }
  std::vector<int> vexcl(Vtot, 0);
  for (OrderDesc& od : pl->items) {
    const int d = od.d;
    int Esum = 0;
    if (dwp) {
      std::vector<int> sig(od.R, 0);
      for (int r = 0; r < od.R; ++r)
        for (int m = 0; m < d; ++m) sig[r] += ev[od.vbase + m * od.R + r];
      Esum = *std::max_element(sig.begin(), sig.end());
      std::vector<float> rs(od.R);
      for (int r = 0; r < od.R; ++r) rs[r] = std::ldexp(1.0f, sig[r] - Esum);
      if ((e = cudaMemcpy((void*)od.rscale, rs.data(), sizeof(float) * od.R, cudaMemcpyHostToDevice)) !=
          cudaSuccess)
        return cuda_fail(e, "upload rank scales");
    }
    od.pscale = std::ldexp(1.0, Esum - d) / ((double)od.L * factorial(d));
    for (int m = 0; m < d; ++m)
      for (int r = 0; r < od.R; ++r) {
        int sum = 0;
        for (int mm = 0; mm < d; ++mm)
          if (mm != m) sum += ev[od.vbase + mm * od.R + r];
        vexcl[od.vbase + m * od.R + r] = sum;
      }
  }
  if ((e = cudaMemcpy((void*)P.ord, pl->items.data(), sizeof(OrderDesc) * pl->items.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy((void*)P.vexcl, vexcl.data(), sizeof(int) * Vtot, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "upload tables");
  return SAG_OK;
}

}  // namespace sag
