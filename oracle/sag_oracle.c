/*
 * CPU oracle for the multi-particle Smoluchowski right-hand side.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg, never by the library. It shares no code with
 * the CUDA path. Everything is FP64; sums that run over many terms use
 * Neumaier's compensated summation so that the oracle's own rounding stays far
 * below the tolerances it is used to check.
 *
 * Two evaluation modes, both written from the definitions in Sec. 1:
 *   ORC_BRUTE  - enumerate every index tuple, O(N^d) per order d;
 *   ORC_DIRECT - the low-rank route without any FFT: for CP (Sec. 1, "pre-defined
 *                low-rank CP") each rank term is a sequential d-fold linear
 *                convolution of the vectors U^(m)_r o n; for TT (Eq. ch3.eq4) the
 *                same with matrix-valued vectors. Q uses inner products.
 * The paper's FFT route computes the same quantity, so the two modes must agree
 * to rounding with each other and with the GPU library.
 *
 * Readings taken where the paper is silent (each listed in the design notes):
 *   - truncation: every index runs over sizes 1..N; P drops tuples whose sizes
 *     sum past N, Q sums over all of [1,N]^{d-1};
 *   - Q for a non-symmetric kernel: sym = 1 uses the mode-symmetrised kernel
 *     (the paper assumes symmetric coefficients, Sec. 1), sym = 0 puts k in the
 *     last mode exactly as printed;
 *   - the RK2 variant is Heun's method (explicit trapezoid) by default.
 */
#include "sag_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

#define ORC_MAXD 8

/* ---- compensated summation (Neumaier's variant of Kahan's method) ---- */
typedef struct { double s, c; } nsum;
static void ns_add(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double ns_val(const nsum* a) { return a->s + a->c; }

static double factorial(int d) {
  double f = 1.0;
  for (int i = 2; i <= d; ++i) f *= i;
  return f;
}

/* ---- factor layout helpers ---- */
static int ranks_ok(int fmt, int D, int N, const int* ranks) {
  if (D < 2 || D > ORC_MAXD || N < 1 || !ranks) return 0;
  if (fmt == ORC_CP) {
    /* rank 0: the order is absent (its sums over r are empty) */
    for (int d = 2; d <= D; ++d)
      if (ranks[d - 2] < 0) return 0;
    return 1;
  }
  if (fmt == ORC_TT) {
    const int* rk = ranks;
    for (int d = 2; d <= D; ++d) {
      if (rk[0] != 1 || rk[d] != 1) return 0;
      for (int l = 0; l <= d; ++l)
        if (rk[l] < 1) return 0;
      rk += d + 1;
    }
    return 1;
  }
  return 0;
}

/* Offset (in doubles) of order d's block, and the pointer to its ranks. */
static long order_offset(int fmt, int N, const int* ranks, int d, const int** rk_out) {
  long off = 0;
  const int* rk = ranks;
  for (int e = 2; e < d; ++e) {
    if (fmt == ORC_CP) {
      off += (long)e * rk[0] * N;
      rk += 1;
    } else {
      for (int l = 1; l <= e; ++l) off += (long)rk[l - 1] * rk[l] * N;
      rk += e + 1;
    }
  }
  if (rk_out) *rk_out = rk;
  return off;
}

long orc_factor_count(int fmt, int D, int N, const int* ranks) {
  if (!ranks_ok(fmt, D, N, ranks)) return -1;
  return order_offset(fmt, N, ranks, D + 1, NULL);
}

/* CP vector U^(m)_r of order d (m, r 0-based). */
static const double* cp_vec(const double* blk, int R, int N, int m, int r) {
  return blk + ((long)m * R + r) * N;
}
/* TT vector h^(lambda)_{a,b} of order d (lambda 1-based, a, b 0-based). */
static const double* tt_vec(const double* blk, const int* rk, int N, int lambda, int a, int b) {
  long off = 0;
  for (int l = 1; l < lambda; ++l) off += (long)rk[l - 1] * rk[l] * N;
  return blk + off + ((long)a * rk[lambda] + b) * N;
}

/* Kernel element from its factors: CP sum of rank-one products (Sec. 1), or
 * the TT matrix product of Eq. ch3.eq4. idx holds 1-based sizes. */
static double entry_blk(int fmt, int N, const int* rk, const double* blk, int d, const int* idx) {
  if (fmt == ORC_CP) {
    const int R = rk[0];
    double acc = 0.0;
    for (int r = 0; r < R; ++r) {
      double prod = 1.0;
      for (int m = 0; m < d; ++m) prod *= cp_vec(blk, R, N, m, r)[idx[m] - 1];
      acc += prod;
    }
    return acc;
  }
  /* TT: row vector v (length R_lambda) times core slices H^(lambda)(i_lambda). */
  double v[128], w[128];
  int len = 1;
  v[0] = 1.0;
  for (int l = 1; l <= d; ++l) {
    const int ra = rk[l - 1], rb = rk[l];
    for (int b = 0; b < rb; ++b) {
      double acc = 0.0;
      for (int a = 0; a < ra; ++a) acc += v[a] * tt_vec(blk, rk, N, l, a, b)[idx[l - 1] - 1];
      w[b] = acc;
    }
    len = rb;
    memcpy(v, w, sizeof(double) * len);
  }
  return v[0];
}

double orc_kernel_entry(int fmt, int D, int N, const int* ranks, const double* factors, int d,
                        const int* idx) {
  if (!ranks_ok(fmt, D, N, ranks) || d < 2 || d > D) return NAN;
  const int* rk;
  long off = order_offset(fmt, N, ranks, d, &rk);
  return entry_blk(fmt, N, rk, factors + off, d, idx);
}

/* ---------------------------------------------------------------------------
 * Brute force: enumerate tuples exactly as the definitions of p_k^(d) and
 * q_k^(d) in Sec. 1 read.
 * ------------------------------------------------------------------------- */

/* All permutations of 0..d-1 in lexicographic order; returns their count. */
static int all_perms(int d, int* out /* [d!][d] */) {
  int a[ORC_MAXD];
  for (int i = 0; i < d; ++i) a[i] = i;
  int cnt = 0;
  for (;;) {
    memcpy(out + (long)cnt * d, a, sizeof(int) * d);
    ++cnt;
    int i = d - 2;
    while (i >= 0 && a[i] > a[i + 1]) --i;
    if (i < 0) break;
    int j = d - 1;
    while (a[j] < a[i]) --j;
    int t = a[i]; a[i] = a[j]; a[j] = t;
    for (int l = i + 1, h = d - 1; l < h; ++l, --h) { t = a[l]; a[l] = a[h]; a[h] = t; }
  }
  return cnt;
}

/* Advance a 1-based odometer over [1,N]^len; returns 0 when it wraps. */
static int odometer_next(int* idx, int len, int N) {
  for (int p = len - 1; p >= 0; --p) {
    if (idx[p] < N) { ++idx[p]; return 1; }
    idx[p] = 1;
  }
  return 0;
}

static void rhs_brute_order(int fmt, int N, const int* rk, const double* blk, int d,
                            const double* n, int sym, nsum* p, nsum* q, nsum* out) {
  const double inv_dfact = 1.0 / factorial(d);
  const double inv_d1fact = 1.0 / factorial(d - 1);
  int idx[ORC_MAXD];
  /* P^(d) and the outflow: every ordered d-tuple in [1,N]^d. */
  for (int m = 0; m < d; ++m) idx[m] = 1;
  do {
    int k = 0;
    double w = entry_blk(fmt, N, rk, blk, d, idx);
    for (int m = 0; m < d; ++m) { k += idx[m]; w *= n[idx[m] - 1]; }
    if (k <= N) ns_add(&p[k - 1], w * inv_dfact);
    else if (out) ns_add(out, (double)k * w * inv_dfact);
  } while (odometer_next(idx, d, N));

  /* Q^(d): k fixed, the other d-1 indices over [1,N]^{d-1}. */
  int nperm = 1;
  int* perms = NULL;
  if (sym) {
    for (int i = 2; i <= d; ++i) nperm *= i;
    perms = (int*)malloc(sizeof(int) * nperm * d);
    all_perms(d, perms);
  }
  for (int k = 1; k <= N; ++k) {
    nsum acc = {0.0, 0.0};
    for (int m = 0; m < d - 1; ++m) idx[m] = 1;
    do {
      int full[ORC_MAXD], pidx[ORC_MAXD];
      for (int m = 0; m < d - 1; ++m) full[m] = idx[m];
      full[d - 1] = k;
      double c;
      if (sym) {
        /* C_sym = average of C over all orderings of its d modes. */
        double cs = 0.0;
        for (int s = 0; s < nperm; ++s) {
          for (int m = 0; m < d; ++m) pidx[m] = full[perms[s * d + m]];
          cs += entry_blk(fmt, N, rk, blk, d, pidx);
        }
        c = cs / nperm;
      } else {
        c = entry_blk(fmt, N, rk, blk, d, full);
      }
      double w = c;
      for (int m = 0; m < d - 1; ++m) w *= n[idx[m] - 1];
      ns_add(&acc, w);
    } while (d > 1 && odometer_next(idx, d - 1, N));
    ns_add(&q[k - 1], -n[k - 1] * inv_d1fact * ns_val(&acc));
  }
  free(perms);
}

/* ---------------------------------------------------------------------------
 * Direct low-rank evaluation (no FFT).
 * ------------------------------------------------------------------------- */

/* Linear convolution of b (sizes 1..lb) with a (sizes 1..N), written for sizes
 * 1..lc: c[k] = sum_{i + j = k} b[i] a[j]. Arrays are 1-based by size (index
 * k-1). Sums are compensated. */
static void conv_sizes(const double* b, int lb, const double* a, int N, double* c, int lc) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int k = 1; k <= lc; ++k) {
    nsum acc = {0.0, 0.0};
    int ilo = k - N > 1 ? k - N : 1;
    int ihi = k - 1 < lb ? k - 1 : lb;
    for (int i = ilo; i <= ihi; ++i) ns_add(&acc, b[i - 1] * a[k - i - 1]);
    c[k - 1] = ns_val(&acc);
  }
}

static double dot_n(const double* u, const double* n, int N) {
  nsum acc = {0.0, 0.0};
  for (int k = 0; k < N; ++k) ns_add(&acc, u[k] * n[k]);
  return ns_val(&acc);
}

/* Adds the finished d-fold convolution g (sizes 1..lg) into P and the outflow. */
static void scatter_gain(const double* g, int lg, int N, double inv_dfact, nsum* p, nsum* out) {
  for (int k = 1; k <= lg; ++k) {
    if (k <= N) ns_add(&p[k - 1], g[k - 1] * inv_dfact);
    else if (out) ns_add(out, (double)k * g[k - 1] * inv_dfact);
  }
}

static void gain_cp_order(int N, int R, const double* blk, int d, const double* n, nsum* p,
                          nsum* out) {
  const double inv_dfact = 1.0 / factorial(d);
  const int Lmax = out ? d * N : N;
  double* a = (double*)malloc(sizeof(double) * N);
  double* b = (double*)malloc(sizeof(double) * Lmax);
  double* c = (double*)malloc(sizeof(double) * Lmax);
  for (int r = 0; r < R; ++r) {
    /* Gain: a^(1) * a^(2) * ... * a^(d), a^(m) = U^(m)_r o n. */
    const double* u1 = cp_vec(blk, R, N, 0, r);
    int lb = N;
    for (int k = 0; k < N; ++k) b[k] = u1[k] * n[k];
    for (int m = 1; m < d; ++m) {
      const double* um = cp_vec(blk, R, N, m, r);
      for (int k = 0; k < N; ++k) a[k] = um[k] * n[k];
      int lc = out ? (m + 1) * N : N;
      conv_sizes(b, lb, a, N, c, lc);
      memcpy(b, c, sizeof(double) * lc);
      lb = lc;
    }
    scatter_gain(b, lb, N, inv_dfact, p, out);
  }
  free(a); free(b); free(c);
}

/* Loss of a CP order: s_m = <U^(m)_r, n>; the kernel row through k is a sum
 * over the position k takes (sym) or the last mode only (literal). */
static void loss_cp_order(int N, int R, const double* blk, int d, const double* n, int sym,
                          nsum* q) {
  const double inv_d1fact = 1.0 / factorial(d - 1);
  double* s = (double*)malloc(sizeof(double) * d);
  double* w = (double*)calloc(N, sizeof(double));
  for (int r = 0; r < R; ++r) {
    for (int m = 0; m < d; ++m) s[m] = dot_n(cp_vec(blk, R, N, m, r), n, N);
    for (int m = (sym ? 0 : d - 1); m < d; ++m) {
      double coef = 1.0;
      for (int mm = 0; mm < d; ++mm)
        if (mm != m) coef *= s[mm];
      if (sym) coef /= d;
      const double* um = cp_vec(blk, R, N, m, r);
      for (int k = 0; k < N; ++k) w[k] += coef * um[k];
    }
  }
  for (int k = 0; k < N; ++k) ns_add(&q[k], -n[k] * inv_d1fact * w[k]);
  free(s); free(w);
}

static void gain_tt_order(int N, const int* rk, const double* blk, int d, const double* n, nsum* p,
                          nsum* out) {
  const double inv_dfact = 1.0 / factorial(d);
  const int Lmax = out ? d * N : N;
  int rmax = 1;
  for (int l = 0; l <= d; ++l) rmax = rk[l] > rmax ? rk[l] : rmax;
  /* Gain: V_1[b] = h^(1)_{0,b} o n; V_l[b] = sum_a V_{l-1}[a] * (h^(l)_{a,b} o n). */
  double* V = (double*)calloc((size_t)rmax * Lmax, sizeof(double));
  double* W = (double*)calloc((size_t)rmax * Lmax, sizeof(double));
  double* a = (double*)malloc(sizeof(double) * N);
  double* c = (double*)malloc(sizeof(double) * Lmax);
  int lv = N;
  for (int b = 0; b < rk[1]; ++b) {
    const double* h = tt_vec(blk, rk, N, 1, 0, b);
    for (int k = 0; k < N; ++k) V[(size_t)b * Lmax + k] = h[k] * n[k];
  }
  for (int l = 2; l <= d; ++l) {
    int lw = out ? l * N : N;
    for (int b = 0; b < rk[l]; ++b) {
      double* wb = W + (size_t)b * Lmax;
      for (int k = 0; k < lw; ++k) wb[k] = 0.0;
      for (int aa = 0; aa < rk[l - 1]; ++aa) {
        const double* h = tt_vec(blk, rk, N, l, aa, b);
        for (int k = 0; k < N; ++k) a[k] = h[k] * n[k];
        conv_sizes(V + (size_t)aa * Lmax, lv, a, N, c, lw);
        for (int k = 0; k < lw; ++k) wb[k] += c[k];
      }
    }
    double* t = V; V = W; W = t;
    lv = lw;
  }
  scatter_gain(V, lv, N, inv_dfact, p, out);
  free(V); free(W); free(a); free(c);
}

/* Loss of a TT order: M_l = sum_i n_i H^(l)(i) (R_{l-1} x R_l); for k at
 * position pos the kernel sum is M_1 ... M_{pos-1} H^(pos)(k) M_{pos+1} ... M_d. */
static void loss_tt_order(int N, const int* rk, const double* blk, int d, const double* n, int sym,
                          nsum* q) {
  const double inv_d1fact = 1.0 / factorial(d - 1);
  int rmax = 1;
  for (int l = 0; l <= d; ++l) rmax = rk[l] > rmax ? rk[l] : rmax;
  double* M = (double*)malloc(sizeof(double) * (size_t)d * rmax * rmax);
  for (int l = 1; l <= d; ++l)
    for (int aa = 0; aa < rk[l - 1]; ++aa)
      for (int b = 0; b < rk[l]; ++b)
        M[((size_t)(l - 1) * rmax + aa) * rmax + b] = dot_n(tt_vec(blk, rk, N, l, aa, b), n, N);
  double* wsum = (double*)calloc(N, sizeof(double));
  double left[128], right[128], tmp[128];
  for (int pos = (sym ? 1 : d); pos <= d; ++pos) {
    /* left = e_0^T M_1 ... M_{pos-1} (length R_{pos-1}) */
    left[0] = 1.0;
    for (int l = 1; l < pos; ++l) {
      for (int b = 0; b < rk[l]; ++b) {
        double acc = 0.0;
        for (int aa = 0; aa < rk[l - 1]; ++aa) acc += left[aa] * M[((size_t)(l - 1) * rmax + aa) * rmax + b];
        tmp[b] = acc;
      }
      memcpy(left, tmp, sizeof(double) * rk[l]);
    }
    /* right = M_{pos+1} ... M_d e_0 (length R_pos) */
    right[0] = 1.0;
    for (int l = d; l > pos; --l) {
      for (int aa = 0; aa < rk[l - 1]; ++aa) {
        double acc = 0.0;
        for (int b = 0; b < rk[l]; ++b) acc += M[((size_t)(l - 1) * rmax + aa) * rmax + b] * right[b];
        tmp[aa] = acc;
      }
      memcpy(right, tmp, sizeof(double) * rk[l - 1]);
    }
    const double wt = sym ? 1.0 / d : 1.0;
    for (int aa = 0; aa < rk[pos - 1]; ++aa)
      for (int b = 0; b < rk[pos]; ++b) {
        const double coef = wt * left[aa] * right[b];
        const double* h = tt_vec(blk, rk, N, pos, aa, b);
        for (int k = 0; k < N; ++k) wsum[k] += coef * h[k];
      }
  }
  for (int k = 0; k < N; ++k) ns_add(&q[k], -n[k] * inv_d1fact * wsum[k]);
  free(M); free(wsum);
}

int orc_rhs(int mode, int fmt, int D, int N, const int* ranks, const double* factors,
            const double* n, int sym, double* p, double* q, double* outflow) {
  if (!ranks_ok(fmt, D, N, ranks) || !factors || !n || !p || !q) return -1;
  if (mode != ORC_BRUTE && mode != ORC_DIRECT) return -1;
  if (fmt == ORC_TT) {
    const int* rk = ranks;
    for (int d = 2; d <= D; ++d) {
      for (int l = 0; l <= d; ++l)
        if (rk[l] > 128) return -1;
      rk += d + 1;
    }
  }
  nsum* ps = (nsum*)calloc(N, sizeof(nsum));
  nsum* qs = (nsum*)calloc(N, sizeof(nsum));
  nsum os = {0.0, 0.0};
  for (int d = 2; d <= D; ++d) {
    const int* rk;
    const double* blk = factors + order_offset(fmt, N, ranks, d, &rk);
    if (mode == ORC_BRUTE)
      rhs_brute_order(fmt, N, rk, blk, d, n, sym, ps, qs, outflow ? &os : NULL);
    else if (fmt == ORC_CP) {
      gain_cp_order(N, rk[0], blk, d, n, ps, outflow ? &os : NULL);
      loss_cp_order(N, rk[0], blk, d, n, sym, qs);
    } else {
      gain_tt_order(N, rk, blk, d, n, ps, outflow ? &os : NULL);
      loss_tt_order(N, rk, blk, d, n, sym, qs);
    }
  }
  for (int k = 0; k < N; ++k) { p[k] = ns_val(&ps[k]); q[k] = ns_val(&qs[k]); }
  if (outflow) *outflow = ns_val(&os);
  free(ps); free(qs);
  return 0;
}

static int tt_ranks_small(int fmt, int D, const int* ranks) {
  if (fmt != ORC_TT) return 1;
  const int* rk = ranks;
  for (int d = 2; d <= D; ++d) {
    for (int l = 0; l <= d; ++l)
      if (rk[l] > 128) return 0;
    rk += d + 1;
  }
  return 1;
}

int orc_loss(int fmt, int D, int N, const int* ranks, const double* factors, const double* n,
             int sym, double* q) {
  if (!ranks_ok(fmt, D, N, ranks) || !factors || !n || !q || !tt_ranks_small(fmt, D, ranks)) return -1;
  nsum* qs = (nsum*)calloc(N, sizeof(nsum));
  for (int d = 2; d <= D; ++d) {
    const int* rk;
    const double* blk = factors + order_offset(fmt, N, ranks, d, &rk);
    if (fmt == ORC_CP) loss_cp_order(N, rk[0], blk, d, n, sym, qs);
    else loss_tt_order(N, rk, blk, d, n, sym, qs);
  }
  for (int k = 0; k < N; ++k) q[k] = ns_val(&qs[k]);
  free(qs);
  return 0;
}

/* ---------------------------------------------------------------------------
 * Time integration: the explicit second-order Runge-Kutta step of Sec. 3
 * (two right-hand-side evaluations per step).
 * ------------------------------------------------------------------------- */
static void moments(const double* n, int N, double* m0, double* m1) {
  nsum a = {0.0, 0.0}, b = {0.0, 0.0};
  for (int k = 0; k < N; ++k) { ns_add(&a, n[k]); ns_add(&b, (double)(k + 1) * n[k]); }
  *m0 = ns_val(&a);
  *m1 = ns_val(&b);
}

int orc_integrate(int mode, int fmt, int D, int N, const int* ranks, const double* factors,
                  double* n, double dt, long steps, int sym, int method, double* diag) {
  if (!ranks_ok(fmt, D, N, ranks) || !factors || !n || steps < 0) return -1;
  if (method != ORC_HEUN && method != ORC_MIDPOINT) return -1;
  double* p = (double*)malloc(sizeof(double) * N);
  double* q = (double*)malloc(sizeof(double) * N);
  double* k1 = (double*)malloc(sizeof(double) * N);
  double* ns = (double*)malloc(sizeof(double) * N);
  double cum = 0.0, o1 = 0.0, o2 = 0.0;
  double* op = diag ? &o1 : NULL;
  int rc = 0;
  if (diag) { moments(n, N, &diag[0], &diag[1]); diag[2] = 0.0; }
  for (long s = 0; s < steps && rc == 0; ++s) {
    rc = orc_rhs(mode, fmt, D, N, ranks, factors, n, sym, p, q, op);
    for (int k = 0; k < N; ++k) k1[k] = p[k] + q[k];
    const double h1 = method == ORC_HEUN ? dt : 0.5 * dt;
    for (int k = 0; k < N; ++k) ns[k] = n[k] + h1 * k1[k];
    if (rc == 0) rc = orc_rhs(mode, fmt, D, N, ranks, factors, ns, sym, p, q, diag ? &o2 : NULL);
    if (method == ORC_HEUN) {
      /* Heun: n <- n + dt/2 (F(n) + F(n + dt F(n))). */
      for (int k = 0; k < N; ++k) n[k] = n[k] + 0.5 * dt * (k1[k] + (p[k] + q[k]));
      cum += 0.5 * dt * (o1 + o2);
    } else {
      /* Midpoint: n <- n + dt F(n + dt/2 F(n)). */
      for (int k = 0; k < N; ++k) n[k] = n[k] + dt * (p[k] + q[k]);
      cum += dt * o2;
    }
    if (diag) {
      double* row = diag + 3 * (s + 1);
      moments(n, N, &row[0], &row[1]);
      row[2] = cum;
    }
  }
  free(p); free(q); free(k1); free(ns);
  return rc;
}

/* ---------------------------------------------------------------------------
 * Generalized Brownian kernel (Eq. ch3.eq17) and its TT cores (Theorem 1).
 * ------------------------------------------------------------------------- */
double orc_brownian_entry(int D, const double* mu, const int* idx) {
  if (D < 1 || D > ORC_MAXD) return NAN;
  int cnt = 1;
  for (int i = 2; i <= D; ++i) cnt *= i;
  int* perms = (int*)malloc(sizeof(int) * cnt * D);
  all_perms(D, perms);
  double acc = 0.0;
  for (int s = 0; s < cnt; ++s) {
    double prod = 1.0;
    for (int m = 0; m < D; ++m) prod *= pow((double)idx[perms[s * D + m]], mu[m]);
    acc += prod;
  }
  free(perms);
  return acc;
}

static int popcount_int(unsigned x) {
  int c = 0;
  while (x) { c += x & 1u; x >>= 1; }
  return c;
}
static long binom_l(int n, int k) {
  long b = 1;
  for (int i = 1; i <= k; ++i) b = b * (n - k + i) / i;
  return b;
}
/* The rank index r_lambda <-> lambda-subset bijection: subsets of {0..D-1} as
 * bit masks with lambda bits set, in increasing numeric order. */
static int subsets_of_size(int D, int lambda, unsigned* out) {
  int c = 0;
  for (unsigned m = 0; m < (1u << D); ++m)
    if (popcount_int(m) == lambda) out[c++] = m;
  return c;
}

long orc_brownian_tt_count(int D, int N) {
  if (D < 2 || D > ORC_MAXD || N < 1) return -1;
  long tot = 0;
  for (int l = 1; l <= D; ++l) tot += binom_l(D, l - 1) * binom_l(D, l) * N;
  return tot;
}

int orc_brownian_tt(int D, int N, const double* mu, int* ranks_out, double* cores_out) {
  if (D < 2 || D > ORC_MAXD || N < 1 || !mu || !ranks_out || !cores_out) return -1;
  unsigned prev[256], cur[256];
  for (int l = 0; l <= D; ++l) ranks_out[l] = (int)binom_l(D, l);
  int np = subsets_of_size(D, 0, prev); /* the empty set, r_0 = 1 */
  double* out = cores_out;
  for (int l = 1; l <= D; ++l) {
    int nc = subsets_of_size(D, l, cur);
    /* H^(l)[a, i, b] = i^{mu_j} when subset(b) = subset(a) + {j}, else 0. The
     * base case l = 1 is H^(1)[0, i, b] = i^{mu_j} with subset(b) = {j}. */
    for (int a = 0; a < np; ++a)
      for (int b = 0; b < nc; ++b) {
        double* v = out + ((long)a * nc + b) * N;
        unsigned diff = cur[b] & ~prev[a];
        int ok = (prev[a] & ~cur[b]) == 0 && popcount_int(diff) == 1;
        int j = 0;
        while (ok && !((diff >> j) & 1u)) ++j;
        for (int i = 1; i <= N; ++i) v[i - 1] = ok ? pow((double)i, mu[j]) : 0.0;
      }
    out += (long)np * nc * N;
    memcpy(prev, cur, sizeof(unsigned) * nc);
    np = nc;
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Discrete adjoint (vector-Jacobian products), CP kernels. Written from the
 * definitions of p_k^(d) and q_k^(d) (Sec. 1) by the product rule:
 *   d p_k / d a^(m)_r[i] = 1/d! (conv_{m' != m} a^(m')_r)[k - i],
 * so the cotangent of a^(m)_r is the correlation of g with the other modes'
 * convolution, and a^(m)_r = U^(m)_r o n passes it to n and to U; the loss
 * term q_k = n_k sum_v coef_v U_v(k) is differentiated through n_k, through
 * U_v(k) and through the inner products s inside coef.
 * ------------------------------------------------------------------------- */
static void vjp_cp_order(int N, int R, const double* blk, int d, const double* n, const double* g,
                         int sym, double* gn, double* gblk) {
  const double inv_dfact = 1.0 / factorial(d);
  const double inv_d1fact = 1.0 / factorial(d - 1);
  double* a = (double*)malloc(sizeof(double) * (size_t)d * N);
  double* c = (double*)malloc(sizeof(double) * N);
  double* t = (double*)malloc(sizeof(double) * N);
  double* s = (double*)malloc(sizeof(double) * d);
  double* z = (double*)malloc(sizeof(double) * d);
  double* gn_n = (double*)malloc(sizeof(double) * N);
  for (int k = 0; k < N; ++k) gn_n[k] = g[k] * n[k];
  for (int r = 0; r < R; ++r) {
    for (int m = 0; m < d; ++m) {
      const double* u = cp_vec(blk, R, N, m, r);
      for (int k = 0; k < N; ++k) a[(size_t)m * N + k] = u[k] * n[k];
    }
    /* Gain. */
    for (int m = 0; m < d; ++m) {
      /* c = convolution of every other mode, sizes 1..N */
      int first = 1;
      for (int mm = 0; mm < d; ++mm) {
        if (mm == m) continue;
        if (first) {
          memcpy(c, a + (size_t)mm * N, sizeof(double) * N);
          first = 0;
        } else {
          conv_sizes(c, N, a + (size_t)mm * N, N, t, N);
          memcpy(c, t, sizeof(double) * N);
        }
      }
      /* ga[i] = 1/d! sum_{j >= 1, i + j <= N} g[i + j] c[j] (sizes, 1-based) */
      const double* u = cp_vec(blk, R, N, m, r);
      double* gu = gblk + ((size_t)m * R + r) * N;
#pragma omp parallel for schedule(dynamic, 64)
      for (int i = 1; i <= N; ++i) {
        nsum acc = {0.0, 0.0};
        for (int j = 1; i + j <= N; ++j) ns_add(&acc, g[i + j - 1] * c[j - 1]);
        const double ga = inv_dfact * ns_val(&acc);
        gn[i - 1] += u[i - 1] * ga;
        gu[i - 1] += n[i - 1] * ga;
      }
    }
    /* Loss. coef_m = -1/(d-1)! w_m prod_{m' != m} s_{m'}, w_m = 1/d (sym) or [m = d-1]. */
    for (int m = 0; m < d; ++m) {
      s[m] = dot_n(cp_vec(blk, R, N, m, r), n, N);
      z[m] = dot_n(cp_vec(blk, R, N, m, r), gn_n, N);
    }
    for (int m = 0; m < d; ++m) {
      const double wm = sym ? 1.0 / d : (m == d - 1 ? 1.0 : 0.0);
      double coef = -inv_d1fact * wm;
      for (int mm = 0; mm < d; ++mm)
        if (mm != m) coef *= s[mm];
      /* sigma = dL/ds_m: coef_{m2} depends on s_m for every m2 != m */
      double sigma = 0.0;
      for (int m2 = 0; m2 < d; ++m2) {
        if (m2 == m) continue;
        const double w2 = sym ? 1.0 / d : (m2 == d - 1 ? 1.0 : 0.0);
        double p = -inv_d1fact * w2 * z[m2];
        for (int mm = 0; mm < d; ++mm)
          if (mm != m2 && mm != m) p *= s[mm];
        sigma += p;
      }
      const double* u = cp_vec(blk, R, N, m, r);
      double* gu = gblk + ((size_t)m * R + r) * N;
      for (int k = 0; k < N; ++k) {
        gn[k] += g[k] * coef * u[k] + sigma * u[k];
        gu[k] += coef * g[k] * n[k] + sigma * n[k];
      }
    }
  }
  free(a); free(c); free(t); free(s); free(z); free(gn_n);
}

/* Vector-Jacobian product of a TT order (Eq. ch3.eq4), by the chain rule
 * through the same sequence of operations the direct mode evaluates.
 * Gain: A_l[a,b] = h^(l)_{a,b} o n; V_1[b] = A_1[0,b]; V_l[b] = sum_a
 * V_{l-1}[a] * A_l[a,b] (truncated convolutions); p = V_d[0] / d!. Going
 * back with G_d[0] = g / d!: the cotangent of A_l[a,b] is the correlation of
 * G_l[b] with V_{l-1}[a] (l >= 2; G_1[b] itself for l = 1), and G_{l-1}[a] =
 * sum_b the correlation of G_l[b] with A_l[a,b]; A = h o n passes each
 * cotangent to h (times n) and to n (times h).
 * Loss: q_k = c n_k w_k with c = -1/(d-1)!, w_k = sum_pos wt_pos
 * left_{pos-1} H^(pos)(k) right_{pos+1}, left/right the products of the
 * matrices M_l = sum_i n_i H^(l)(i) before and after position pos (as in
 * loss_tt_order). Directly, g.q depends on n_k and H^(pos)(k); through M_l
 * it is, for each pos, the chain e_0^T X_1 ... X_d e_0 with X_pos = z_pos =
 * sum_k g_k n_k H^(pos)(k) and X_l = M_l elsewhere, whose derivative with
 * respect to X_l is the outer product of the chain's prefix before l and
 * suffix after l. */
static void chain_prefix(int d, const int* rk, const double* X, int rmax, int upto, double* out) {
  /* out = e_0^T X_1 ... X_upto (length rk[upto]); X_l at X + (l-1) rmax^2 */
  double tmp[128];
  out[0] = 1.0;
  for (int l = 1; l <= upto; ++l) {
    const double* Xl = X + (size_t)(l - 1) * rmax * rmax;
    for (int b = 0; b < rk[l]; ++b) {
      double acc = 0.0;
      for (int a = 0; a < rk[l - 1]; ++a) acc += out[a] * Xl[(size_t)a * rmax + b];
      tmp[b] = acc;
    }
    memcpy(out, tmp, sizeof(double) * rk[l]);
  }
  (void)d;
}
static void chain_suffix(int d, const int* rk, const double* X, int rmax, int from, double* out) {
  /* out = X_from ... X_d e_0 (length rk[from - 1]) */
  double tmp[128];
  out[0] = 1.0;
  for (int l = d; l >= from; --l) {
    const double* Xl = X + (size_t)(l - 1) * rmax * rmax;
    for (int a = 0; a < rk[l - 1]; ++a) {
      double acc = 0.0;
      for (int b = 0; b < rk[l]; ++b) acc += Xl[(size_t)a * rmax + b] * out[b];
      tmp[a] = acc;
    }
    memcpy(out, tmp, sizeof(double) * rk[l - 1]);
  }
}

static void vjp_tt_order(int N, const int* rk, const double* blk, int d, const double* n, const double* g,
                         int sym, double* gn, double* gblk) {
  const double inv_dfact = 1.0 / factorial(d);
  const double c = -1.0 / factorial(d - 1);
  int rmax = 1;
  for (int l = 0; l <= d; ++l) rmax = rk[l] > rmax ? rk[l] : rmax;
  /* ---- gain: the forward chain, every V_l kept */
  double* V = (double*)calloc((size_t)d * rmax * N, sizeof(double)); /* V_l[b] at ((l-1) rmax + b) N */
  double* a = (double*)malloc(sizeof(double) * N);
  double* t = (double*)malloc(sizeof(double) * N);
  for (int b = 0; b < rk[1]; ++b) {
    const double* h = tt_vec(blk, rk, N, 1, 0, b);
    for (int k = 0; k < N; ++k) V[(size_t)b * N + k] = h[k] * n[k];
  }
  for (int l = 2; l <= d; ++l)
    for (int b = 0; b < rk[l]; ++b) {
      double* vb = V + ((size_t)(l - 1) * rmax + b) * N;
      for (int aa = 0; aa < rk[l - 1]; ++aa) {
        const double* h = tt_vec(blk, rk, N, l, aa, b);
        for (int k = 0; k < N; ++k) a[k] = h[k] * n[k];
        conv_sizes(V + ((size_t)(l - 2) * rmax + aa) * N, N, a, N, t, N);
        for (int k = 0; k < N; ++k) vb[k] += t[k];
      }
    }
  /* ---- gain: back through the chain */
  double* G = (double*)calloc((size_t)rmax * N, sizeof(double));
  double* Gp = (double*)calloc((size_t)rmax * N, sizeof(double));
  double* ga = (double*)malloc(sizeof(double) * N);
  for (int k = 0; k < N; ++k) G[k] = g[k] * inv_dfact;
  for (int l = d; l >= 1; --l) {
    for (size_t i = 0; i < (size_t)rmax * N; ++i) Gp[i] = 0.0;
    for (int aa = 0; aa < rk[l - 1]; ++aa)
      for (int b = 0; b < rk[l]; ++b) {
        const double* h = tt_vec(blk, rk, N, l, aa, b);
        double* gh = gblk + (tt_vec(blk, rk, N, l, aa, b) - blk);
        const double* Gb = G + (size_t)b * N;
        if (l == 1) {
          memcpy(ga, Gb, sizeof(double) * N);
        } else {
          const double* Va = V + ((size_t)(l - 2) * rmax + aa) * N;
          /* ga[j] = sum_{i >= 1, i + j <= N} G_b[i + j] V_a[i] (sizes, 1-based) */
#pragma omp parallel for schedule(dynamic, 64)
          for (int j = 1; j <= N; ++j) {
            nsum acc = {0.0, 0.0};
            for (int i = 1; i + j <= N; ++i) ns_add(&acc, Gb[i + j - 1] * Va[i - 1]);
            ga[j - 1] = ns_val(&acc);
          }
          /* G_{l-1}[a][i] += sum_{j >= 1, i + j <= N} G_b[i + j] A[j] */
          for (int k = 0; k < N; ++k) a[k] = h[k] * n[k];
          double* Gpa = Gp + (size_t)aa * N;
#pragma omp parallel for schedule(dynamic, 64)
          for (int i = 1; i <= N; ++i) {
            nsum acc = {0.0, 0.0};
            for (int j = 1; i + j <= N; ++j) ns_add(&acc, Gb[i + j - 1] * a[j - 1]);
            Gpa[i - 1] += ns_val(&acc);
          }
        }
        for (int k = 0; k < N; ++k) {
          gh[k] += ga[k] * n[k];
          gn[k] += ga[k] * h[k];
        }
      }
    double* sw = G;
    G = Gp;
    Gp = sw;
  }
  /* ---- loss */
  const size_t r2 = (size_t)rmax * rmax;
  double* M = (double*)calloc((size_t)d * r2, sizeof(double));
  double* X = (double*)calloc((size_t)d * r2, sizeof(double));
  double* Gam = (double*)calloc((size_t)d * r2, sizeof(double));
  double* gnn = (double*)malloc(sizeof(double) * N);
  double* w = (double*)calloc(N, sizeof(double));
  for (int k = 0; k < N; ++k) gnn[k] = g[k] * n[k];
  for (int l = 1; l <= d; ++l)
    for (int aa = 0; aa < rk[l - 1]; ++aa)
      for (int b = 0; b < rk[l]; ++b)
        M[(l - 1) * r2 + (size_t)aa * rmax + b] = dot_n(tt_vec(blk, rk, N, l, aa, b), n, N);
  double left[128], right[128], pre[128], suf[128];
  for (int pos = (sym ? 1 : d); pos <= d; ++pos) {
    const double wt = sym ? 1.0 / d : 1.0;
    chain_prefix(d, rk, M, rmax, pos - 1, left);
    chain_suffix(d, rk, M, rmax, pos + 1, right);
    /* direct: w_k and the cotangent of H^(pos)(k) */
    for (int aa = 0; aa < rk[pos - 1]; ++aa)
      for (int b = 0; b < rk[pos]; ++b) {
        const double lr = wt * left[aa] * right[b];
        const double* h = tt_vec(blk, rk, N, pos, aa, b);
        double* gh = gblk + (h - blk);
        for (int k = 0; k < N; ++k) {
          w[k] += lr * h[k];
          gh[k] += c * lr * gnn[k];
        }
      }
    /* through M_l, l != pos: the chain with X_pos = z_pos */
    memcpy(X, M, sizeof(double) * (size_t)d * r2);
    for (int aa = 0; aa < rk[pos - 1]; ++aa)
      for (int b = 0; b < rk[pos]; ++b)
        X[(pos - 1) * r2 + (size_t)aa * rmax + b] = dot_n(tt_vec(blk, rk, N, pos, aa, b), gnn, N);
    for (int l = 1; l <= d; ++l) {
      if (l == pos) continue;
      chain_prefix(d, rk, X, rmax, l - 1, pre);
      chain_suffix(d, rk, X, rmax, l + 1, suf);
      for (int aa = 0; aa < rk[l - 1]; ++aa)
        for (int b = 0; b < rk[l]; ++b) Gam[(l - 1) * r2 + (size_t)aa * rmax + b] += c * wt * pre[aa] * suf[b];
    }
  }
  for (int k = 0; k < N; ++k) gn[k] += c * g[k] * w[k];
  for (int l = 1; l <= d; ++l)
    for (int aa = 0; aa < rk[l - 1]; ++aa)
      for (int b = 0; b < rk[l]; ++b) {
        const double gm = Gam[(l - 1) * r2 + (size_t)aa * rmax + b];
        if (gm == 0.0) continue;
        const double* h = tt_vec(blk, rk, N, l, aa, b);
        double* gh = gblk + (h - blk);
        for (int k = 0; k < N; ++k) {
          gn[k] += gm * h[k];
          gh[k] += gm * n[k];
        }
      }
  free(V); free(a); free(t); free(G); free(Gp); free(ga); free(M); free(X); free(Gam); free(gnn); free(w);
}

int orc_rhs_vjp_fmt(int fmt, int D, int N, const int* ranks, const double* factors, const double* n,
                    const double* g, int sym, double* gn, double* gU) {
  if (!ranks_ok(fmt, D, N, ranks) || !factors || !n || !g || !gn || !gU) return -1;
  if (!tt_ranks_small(fmt, D, ranks)) return -1;
  const long nf = orc_factor_count(fmt, D, N, ranks);
  for (int k = 0; k < N; ++k) gn[k] = 0.0;
  for (long i = 0; i < nf; ++i) gU[i] = 0.0;
  for (int d = 2; d <= D; ++d) {
    const int* rk;
    const long off = order_offset(fmt, N, ranks, d, &rk);
    if (fmt == ORC_CP) vjp_cp_order(N, rk[0], factors + off, d, n, g, sym, gn, gU + off);
    else vjp_tt_order(N, rk, factors + off, d, n, g, sym, gn, gU + off);
  }
  return 0;
}

int orc_rhs_vjp(int D, int N, const int* ranks, const double* factors, const double* n,
                const double* g, int sym, double* gn, double* gU) {
  return orc_rhs_vjp_fmt(ORC_CP, D, N, ranks, factors, n, g, sym, gn, gU);
}

/* Reverse pass through `steps` RK2 steps from n0 (states kept in memory).
 * g_in: cotangent of the final state. Outputs g_n0 (cotangent of n0) and g_U
 * (cotangent of the factors, accumulated over all steps). */
int orc_integrate_vjp_fmt(int fmt, int D, int N, const int* ranks, const double* factors, const double* n0,
                          double dt, long steps, int sym, int method, const double* g_in, double* g_n0,
                          double* g_U) {
  if (!ranks_ok(fmt, D, N, ranks) || !factors || !n0 || !g_in || !g_n0 || !g_U || steps < 0)
    return -1;
  if (!tt_ranks_small(fmt, D, ranks)) return -1;
  if (method != ORC_HEUN && method != ORC_MIDPOINT) return -1;
  const long nf = orc_factor_count(fmt, D, N, ranks);
  double* states = (double*)malloc(sizeof(double) * (size_t)(steps + 1) * N);
  double* p = (double*)malloc(sizeof(double) * N);
  double* q = (double*)malloc(sizeof(double) * N);
  double* ns = (double*)malloc(sizeof(double) * N);
  double* gbar = (double*)malloc(sizeof(double) * N);
  double* gk = (double*)malloc(sizeof(double) * N);
  double* gA = (double*)malloc(sizeof(double) * N);
  double* gB = (double*)malloc(sizeof(double) * N);
  double* gUa = (double*)malloc(sizeof(double) * nf);
  memcpy(states, n0, sizeof(double) * N);
  for (long s = 0; s < steps; ++s) {
    memcpy(states + (size_t)(s + 1) * N, states + (size_t)s * N, sizeof(double) * N);
    orc_integrate(ORC_DIRECT, fmt, D, N, ranks, factors, states + (size_t)(s + 1) * N, dt, 1, sym,
                  method, NULL);
  }
  memcpy(gbar, g_in, sizeof(double) * N);
  for (long i = 0; i < nf; ++i) g_U[i] = 0.0;
  for (long s = steps - 1; s >= 0; --s) {
    const double* n = states + (size_t)s * N;
    orc_rhs(ORC_DIRECT, fmt, D, N, ranks, factors, n, sym, p, q, NULL);
    const double h1 = method == ORC_HEUN ? dt : 0.5 * dt;
    for (int k = 0; k < N; ++k) ns[k] = n[k] + h1 * (p[k] + q[k]);
    /* second stage: k2 = F(n*) enters with weight dt/2 (Heun) or dt (midpoint) */
    const double w2 = method == ORC_HEUN ? 0.5 * dt : dt;
    for (int k = 0; k < N; ++k) gk[k] = w2 * gbar[k];
    orc_rhs_vjp_fmt(fmt, D, N, ranks, factors, ns, gk, sym, gA, gUa);
    for (long i = 0; i < nf; ++i) g_U[i] += gUa[i];
    /* first stage: k1 = F(n) enters n' with weight dt/2 (Heun, 0 for midpoint)
     * and n* with weight h1 */
    const double w1 = method == ORC_HEUN ? 0.5 * dt : 0.0;
    for (int k = 0; k < N; ++k) gk[k] = w1 * gbar[k] + h1 * gA[k];
    orc_rhs_vjp_fmt(fmt, D, N, ranks, factors, n, gk, sym, gB, gUa);
    for (long i = 0; i < nf; ++i) g_U[i] += gUa[i];
    for (int k = 0; k < N; ++k) gbar[k] = gbar[k] + gA[k] + gB[k];
  }
  memcpy(g_n0, gbar, sizeof(double) * N);
  free(states); free(p); free(q); free(ns); free(gbar); free(gk); free(gA); free(gB); free(gUa);
  return 0;
}

int orc_integrate_vjp(int D, int N, const int* ranks, const double* factors, const double* n0,
                      double dt, long steps, int sym, int method, const double* g_in, double* g_n0,
                      double* g_U) {
  return orc_integrate_vjp_fmt(ORC_CP, D, N, ranks, factors, n0, dt, steps, sym, method, g_in, g_n0, g_U);
}
