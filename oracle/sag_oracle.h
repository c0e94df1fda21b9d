/*
 * CPU oracle for the multi-particle Smoluchowski right-hand side.
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, slow, FP64 statement of what the
 * GPU library computes. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it. It shares no code, header, table or constant
 * with the CUDA library, and the CUDA library never calls it.
 *
 * Model (paper Sec. 1): dn/dt = sum_{d=2..D} (P^(d)[n] + Q^(d)[n]) with
 *   p_k^(d) = 1/d!     * sum_{i in [1,N]^d, |i| = k} C^(d)_i n_{i_1} ... n_{i_d}
 *   q_k^(d) = -n_k/(d-1)! * sum_{i in [1,N]^{d-1}}  C^(d)_{i,k} n_{i_1} ... n_{i_{d-1}}
 * truncated to sizes k = 1..N (reading: every index runs over 1..N).
 *
 * Conventions shared with the library by interface only:
 *   - size k is stored at array index k-1;
 *   - CP factors of order d: [d][R_d][N] (mode m, rank r, size), orders
 *     d = 2..D concatenated; element C_i = sum_r prod_m U^(m)_r(i_m) (Sec. 1);
 *   - TT cores of order d (Eq. ch3.eq4): for lambda = 1..d a block
 *     [R_{lambda-1}][R_lambda][N], R_0 = R_d = 1, orders concatenated;
 *   - CP ranks: one int per order (R_2..R_D); TT ranks: d+1 ints per order.
 *
 * Every function returns 0 on success and a negative value on bad arguments.
 */
#ifndef SAG_ORACLE_H
#define SAG_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BRUTE = 0, ORC_DIRECT = 1 };   /* evaluation mode */
enum { ORC_CP = 0, ORC_TT = 1 };          /* kernel format */
enum { ORC_HEUN = 0, ORC_MIDPOINT = 1 };  /* explicit second-order Runge-Kutta variant */

/* Threads the OpenMP loops of later calls from this host thread use (n > 0
 * sets it; n <= 0 leaves it); returns the current count. No arithmetic. */
int orc_set_threads(int n);

/* Number of doubles the factor array holds for the given format and ranks. */
long orc_factor_count(int fmt, int D, int N, const int* ranks);

/* One kernel element C^(d)_{i_1..i_d} (1-based sizes in idx). */
double orc_kernel_entry(int fmt, int D, int N, const int* ranks, const double* factors,
                        int d, const int* idx);

/* Right-hand side. p and q (length N each) receive sum_d P^(d) and sum_d Q^(d).
 * sym = 1 evaluates Q for the mode-symmetrised kernel, sym = 0 takes the
 * kernel's last mode literally. outflow (nullable) receives the mass flux out of
 * the truncated system, sum_d 1/d! sum_{i in [1,N]^d, |i| > N} |i| C_i prod n. */
int orc_rhs(int mode, int fmt, int D, int N, const int* ranks, const double* factors,
            const double* n, int sym, double* p, double* q, double* outflow);

/* Loss part only, q = sum_d Q^(d)[n] (length N), in O(N sum_d d R_d) for CP.
 * Same definition and sym flag as orc_rhs. */
int orc_loss(int fmt, int D, int N, const int* ranks, const double* factors, const double* n,
             int sym, double* q);

/* `steps` explicit RK2 steps of size dt on n (in place). diag (nullable)
 * receives [steps+1][3] = (M0, M1, cumulative outflow mass) after each step,
 * row 0 for the initial state. */
int orc_integrate(int mode, int fmt, int D, int N, const int* ranks, const double* factors,
                  double* n, double dt, long steps, int sym, int method, double* diag);

/* Vector-Jacobian product of the right-hand side, CP kernels: for a cotangent
 * g (length N), gn = (dF/dn)^T g and gU = (dF/dU)^T g (factor layout). */
int orc_rhs_vjp(int D, int N, const int* ranks, const double* factors, const double* n,
                const double* g, int sym, double* gn, double* gU);

/* The same for either format (fmt = ORC_CP or ORC_TT; TT cotangents in the
 * core layout). */
int orc_rhs_vjp_fmt(int fmt, int D, int N, const int* ranks, const double* factors, const double* n,
                    const double* g, int sym, double* gn, double* gU);
int orc_integrate_vjp_fmt(int fmt, int D, int N, const int* ranks, const double* factors, const double* n0,
                          double dt, long steps, int sym, int method, const double* g_in, double* g_n0,
                          double* g_U);

/* Discrete adjoint of `steps` RK2 steps from n0, CP kernels: given the
 * cotangent g_in of the final state, returns the cotangent of n0 and the
 * factors' cotangent accumulated over the steps. */
int orc_integrate_vjp(int D, int N, const int* ranks, const double* factors, const double* n0,
                      double dt, long steps, int sym, int method, const double* g_in, double* g_n0,
                      double* g_U);

/* Generalized Brownian kernel entry, Eq. ch3.eq17: sum over permutations sigma
 * of prod_m i_{sigma(m)}^{mu_m}. */
double orc_brownian_entry(int D, const double* mu, const int* idx);

/* TT cores of the generalized Brownian kernel built as in the proof of
 * Theorem 1 (ranks binom(D, lambda)). Writes D+1 ranks to ranks_out and the
 * cores ([R_{l-1}][R_l][N] per lambda, concatenated) to cores_out, which must
 * hold orc_brownian_tt_count(D, N) doubles. */
long orc_brownian_tt_count(int D, int N);
int orc_brownian_tt(int D, int N, const double* mu, int* ranks_out, double* cores_out);

#ifdef __cplusplus
}
#endif
#endif
