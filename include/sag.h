/*
 * sag.h - C ABI of the GB300 library for the multi-particle Smoluchowski
 * right-hand side with low-rank kernels.
 *
 * What it computes (arXiv:1905.09071, Sec. 1): for concentrations n_k of sizes
 * k = 1..N,
 *     dn/dt = sum_{d=2..D} ( P^(d)[n] + Q^(d)[n] ),
 *     p_k^(d) =  1/d!     * sum_{i in [1,N]^d, |i| = k}  C^(d)_i  n_{i_1} ... n_{i_d},
 *     q_k^(d) = -n_k/(d-1)! * sum_{i in [1,N]^{d-1}}      C^(d)_{i,k} n_{i_1} ... n_{i_{d-1}},
 * with every index truncated to 1..N. Each kernel C^(d) is given in low-rank
 * form: CP, C_i = sum_r prod_m U^(m)_r(i_m) (Sec. 1), or TT, Eq. ch3.eq4.
 * The gain P^(d) is evaluated as d-fold truncated convolutions through FFTs,
 * the loss Q^(d) through inner products <U^(m)_r, n> (Sec. 1, complexity
 * O(N D R log N)). Time stepping is the explicit second-order Runge-Kutta
 * method with two right-hand-side evaluations per step (Sec. 3).
 *
 * Conventions of every call:
 *   - Size k of a system is stored at index k-1 of a contiguous FP64 vector.
 *   - Vectors passed to sag_rhs / sag_rk2_step / sag_integrate may live in
 *     device memory or in host memory; host buffers are copied to and from the
 *     device inside the call, on the given stream.
 *   - All calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream). A plan must not be used by two streams at once.
 *   - Argument errors are reported synchronously through the return value and
 *     sag_last_error(); they never launch work. Errors raised on the device
 *     (a non-finite right-hand side) are latched in the plan and reported by
 *     sag_sync_status().
 *   - The caller owns every buffer it passes. sag_plan copies the factors, so
 *     they may be freed when it returns; the plan owns its device workspace.
 */
#ifndef SAG_H
#define SAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sag_plan_s* sag_plan_t;

typedef enum {
  SAG_OK = 0,
  SAG_EINVAL = 1,          /* bad argument (null pointer, size, rank, layout) */
  SAG_ENOMEM = 2,          /* device or host allocation failed */
  SAG_ECUDA = 3,           /* a CUDA runtime call failed (message has the CUDA error) */
  SAG_EUNSUPPORTED = 4,    /* valid request outside what this build implements */
  SAG_ETIMEOUT = 5,        /* a bounded device-side wait expired */
  SAG_ENONFINITE = 6       /* the right-hand side produced Inf or NaN */
} sag_status;

typedef enum { SAG_CP = 0, SAG_TT = 1, SAG_CP_POWER = 2 } sag_format;

/* SAG_FP64: every FFT in FP64.
 * SAG_FP32_SPLIT: FFTs in double-word FP32 (hi + lo pairs); the radix-2/3/4/8
 * butterflies first round their inputs' high words to one grid per butterfly,
 * so that their additions are exact in the high word (about 2^-43 of the
 * butterfly's largest input per rounding; right-hand sides to about 1e-13
 * relative in max-norm).
 * SAG_FP32_SPLIT_EXACT: the same with every butterfly in plain double-word
 * arithmetic (about 2^-47 per value; right-hand sides to about 1e-15), at about
 * 20% lower throughput.
 * The loss inner products, the Runge-Kutta accumulation and the diagnostics
 * stay FP64 in all three. */
typedef enum { SAG_FP64 = 0, SAG_FP32_SPLIT = 1, SAG_FP32_SPLIT_EXACT = 2 } sag_precision;

/* Second-order explicit Runge-Kutta variant (Sec. 3 names the order only):
 * Heun  n+ = n + dt/2 (F(n) + F(n + dt F(n)));
 * midpoint n+ = n + dt F(n + dt/2 F(n)). */
typedef enum { SAG_HEUN = 0, SAG_MIDPOINT = 1 } sag_rk;

/* One system. Orders d = 2..D (2 <= D <= 8), sizes 1..N (N >= 1).
 *   fmt = SAG_CP: rank[d-2] = R_d for d = 2..D; factors holds, for each d in
 *     turn, the array [d][R_d][N] (mode m, rank r, size), i.e. U^(m)_r(k) at
 *     offset_d + (m R_d + r) N + k - 1.
 *   fmt = SAG_TT: for each d in turn, d+1 ranks R_0..R_d with R_0 = R_d = 1
 *     (Eq. ch3.eq4); factors holds, for each d and each core lambda = 1..d,
 *     the array [R_{lambda-1}][R_lambda][N] (the vectors h^(lambda)_{r,r'} of
 *     Sec. 3 stored along the size axis).
 *   fmt = SAG_CP_POWER: a CP kernel whose factors are powers of the size,
 *     U^(m)_r(i) = u i^a (the random power-law workload's form; the
 *     generalized Brownian kernel of Eq. ch3.eq17 is one too): rank as for
 *     SAG_CP; factors holds, for each d in turn, the array [d][R_d][2] of
 *     (u, a) for vector (m, r), with |a| <= 2.5. The plan expands the factors
 *     in FP64 (u pow(i, a)) for the FP64 kernels, and with SAG_FP32_SPLIT the
 *     double-word forward FFT generates u i^a itself (to about 1e-13
 *     relative) instead of reading the factors (the FP64 and
 *     SAG_FP32_SPLIT_EXACT paths read the expanded copies). No
 *     sag_plan_update_factors; the adjoint's factor cotangent is that of the
 *     expanded values.
 * factors_on_device = 1 if `factors` is a device pointer, 0 for host memory. */
typedef struct {
  int32_t N;
  int32_t D;
  int32_t fmt;
  const int32_t* rank;
  const double* factors;
  int32_t factors_on_device;
} sag_system;

typedef struct {
  int32_t prec;          /* sag_precision, default SAG_FP32_SPLIT */
  int32_t rk;            /* sag_rk, default SAG_HEUN */
  int32_t symmetrize_q;  /* 1 (default): loss term of the mode-symmetrised kernel;
                            0: the kernel's last mode holds k, exactly as printed.
                            The two coincide for symmetric kernels (Sec. 1 assumes
                            symmetric coefficients). */
  int32_t autotune;      /* 0 (default): fixed rules. 1: at plan time, time candidates on
                            this plan's own sizes and keep the fastest, each timed as
                            graph-replayed RK2 steps on an internal stream with a
                            synthetic n (synchronising):
                            - the launch layout of the FFT stage: 1 to 4 stream groups
                              of consecutive orders/systems, each a branch of the
                              graph. The results do not depend on this choice;
                            - for a double-word CP plan of 1 to 4 orders, the
                              four-step split of each order's FFT, M = L/2 = M1 M2:
                              the rule's M2 or half of it, where both give compile-
                              time column and row kernels. Whole candidate plans are
                              built, so the plan call takes longer and briefly holds
                              two plans' device memory. The split changes the order of
                              the FFT's roundings, so results differ within the
                              precision's error bound. */
  int32_t max_m2;        /* 0 (default): the rule, M2 = the largest power of two with
                            M2^2 <= M, M2 <= 512 and M2 dividing M. Otherwise a
                            power of two in [4, 512] that caps M2 (shorter rows, longer
                            columns; for tests and tuning). A column length M1 above
                            4096 is SAG_EUNSUPPORTED. */
  const int32_t* m2;     /* NULL (default), or n_m2 host values: the four-step M2 of each
                            order of the plan, in the order sag_plan_describe lists
                            them (systems in turn, orders d = 2..D with a nonzero CP
                            rank; every order of a TT system). 0 keeps the rule for
                            that order; otherwise a power of two in [4, 512] dividing
                            M = L/2, with M1 = M / M2 <= 4096. This reproduces the
                            splits an autotuned plan reports, without tuning again;
                            it replaces max_m2 and the split search. */
  int32_t n_m2;          /* entries of m2: the plan's order count, else SAG_EINVAL */
  int32_t keep_repeats;  /* 0 (default): bitwise-identical factor vectors of a CP order are
                            transformed once (the Brownian kernel's permutations repeat
                            vectors). Such a plan refuses a factor update
                            (sag_plan_update_factors) that makes vectors that were
                            identical at plan time differ. 1: every vector is treated
                            as distinct, for plans whose factors will change (fitting). */
} sag_options;

/* Fills *opt with the defaults. */
void sag_default_options(sag_options* opt);

/* Builds a plan for B independent systems sys[0..B-1] (1 <= B <= 65535; each
 * with its own N, D and ranks; all CP or all TT). Validates the systems,
 * chooses FFT lengths L_d >= d N (products of 2, 3, 5), builds twiddle tables,
 * copies the factors (FP64, plus the double-word copy for SAG_FP32_SPLIT; TT
 * core vectors that are identically zero are skipped) and allocates the
 * workspace. Every kernel of an evaluation then covers all B systems, with one
 * launch per kernel specialisation (column or row length). Limits: N <= 2^22, d N <= 2^24, CP ranks <= 4096, TT ranks <= 16.
 * A CP rank of 0 leaves that order out (for example a purely ternary system:
 * D = 3 with R_2 = 0); every system needs one order of rank >= 1.
 * opt may be NULL (defaults). On success *out holds the plan. */
sag_status sag_plan(const sag_system* sys, int32_t B, const sag_options* opt, sag_plan_t* out);

/* Offsets of each system's block in packed state vectors: offsets[b] is the
 * index of system b's size 1, offsets[B] the total length. `offsets` is a host
 * array of B+1 entries. */
sag_status sag_plan_layout(sag_plan_t plan, int64_t* offsets);

/* Device bytes the plan holds (factor copies, tables, workspace). */
sag_status sag_plan_bytes(sag_plan_t plan, size_t* bytes);

/* dndt = sum_d P^(d)[n] + Q^(d)[n] (Sec. 1). n and dndt hold the packed state
 * (length offsets[B]); they may alias. */
sag_status sag_rhs(sag_plan_t plan, const double* n, double* dndt, void* stream);

/* The gain and loss parts separately: p = sum_d P^(d)[n], q = sum_d Q^(d)[n]
 * (either may be NULL), and outflow[b], b < B (host or device, may be NULL) =
 * the first-moment flux out of truncated system b,
 *     sum_d 1/d! sum_{i in [1,N]^d, |i| > N} |i| C^(d)_i prod_m n_{i_m}. */
sag_status sag_rhs_parts(sag_plan_t plan, const double* n, double* p, double* q,
                         double* outflow, void* stream);

/* One explicit RK2 step of size dt on n, in place (Sec. 3: two right-hand-side
 * evaluations per step). */
sag_status sag_rk2_step(sag_plan_t plan, double* n, double dt, void* stream);

/* One stage of the plan's RK2 rule from a right-hand side k that the caller
 * supplies, for a system whose right-hand side is assembled outside one plan
 * (the term-parallel split: every process evaluates the CP rank terms it owns
 * with sag_rhs and the partial right-hand sides are summed across processes;
 * P and Q are both sums over the terms (d, r), Sec. 1). All vectors are device
 * vectors of the plan's packed length; k may alias neither n, nstar nor k1.
 *   stage 0: k1 = k, nstar = n + h1 k (h1 = dt for Heun, dt/2 for midpoint);
 *            the caller then evaluates k at nstar.
 *   stage 1: Heun n += dt/2 (k1 + k); midpoint n += dt k.
 * A non-finite k latches SAG_ENONFINITE for sag_sync_status. Asynchronous. */
sag_status sag_rk2_stage(sag_plan_t plan, int32_t stage, double* n, double* nstar, double* k1, const double* k,
                         double dt, void* stream);

/* `steps` RK2 steps of size dt on n, in place. The step is captured once as a
 * CUDA graph per (n, dt, diag) and replayed. diag (may be NULL; host or device)
 * receives [steps+1][B][3] doubles: M0 = sum_k n_k, M1 = sum_k k n_k and the
 * cumulative first-moment outflow (the time integral, by the same RK2 rule, of
 * the outflow of sag_rhs_parts); row 0 is the initial state. With a symmetric
 * (or symmetrised) kernel M1 + outflow stays constant. */
sag_status sag_integrate(sag_plan_t plan, double* n, double dt, int64_t steps, double* diag,
                         void* stream);

/* Adjoint (CP and TT plans). The factors' cotangent uses the systems' own
 * factor layout concatenated in system order, sag_plan_factor_count values in
 * all: CP, the arrays [d][R_d][N] per order; TT, the cores
 * [R_{lambda-1}][R_lambda][N] per order (every core entry, also entries whose
 * vector is zero: their cotangents are in general not zero).
 *
 * sag_rhs_vjp: vector-Jacobian product of the right-hand side at n for the
 * cotangent g (packed state layout): gn = (dF/dn)^T g, gU = (dF/dU)^T g
 * (either output may be NULL; both are overwritten). The gain term's
 * derivative is a correlation of g with the other modes' convolution (TT: with
 * the product of the other cores, G conj(prefix[a] suffix[b]) per frequency),
 * evaluated with the same FFT lengths as the forward pass; the loss term's
 * through n, the factors and the inner products s = <U, n> (TT: the matrices
 * M_lambda = sum_i n_i H^(lambda)(i)) by the product rule. */
sag_status sag_rhs_vjp(sag_plan_t plan, const double* n, const double* g, double* gn, double* gU,
                       void* stream);

/* Discrete adjoint of `steps` RK2 steps of size dt from n0 (n0 is not
 * modified): given the cotangent g_final of the final state, writes the
 * cotangent of n0 to g_n0 and the factors' cotangent, summed over the steps,
 * to g_U (either may be NULL). The forward states are recomputed from
 * checkpoints every `ckpt` steps (ckpt <= 0: about sqrt(steps)); device memory
 * for (steps/ckpt + 2 ckpt + 5) state vectors (checkpoints, a segment's states
 * and stage states, work vectors) is allocated on first use. */
sag_status sag_integrate_vjp(sag_plan_t plan, const double* n0, double dt, int64_t steps, int64_t ckpt,
                             const double* g_final, double* g_n0, double* g_U, void* stream);

/* Replaces the factors of a CP plan (same systems and ranks; vector layout as
 * above, host or device pointer) without allocating, so captured graphs stay
 * valid. Synchronises the device first. SAG_EINVAL if the new factors make
 * vectors differ that were bitwise identical when the plan was made (and so
 * share one transform); build such plans with keep_repeats = 1. */
sag_status sag_plan_update_factors(sag_plan_t plan, const double* factors, int32_t on_device);

/* Number of factor values of the plan's systems in their factor layout (the
 * length of the adjoint's factor cotangent). */
sag_status sag_plan_factor_count(sag_plan_t plan, int64_t* count);

/* Clock-cycle limit of the plan's device-side waits (the row kernels' waits on
 * their own bulk copies); cycles <= 0 restores the default, 4e9 (about 2 s at
 * the maximum SM clock). A wait that runs out latches SAG_ETIMEOUT for
 * sag_sync_status, lets the block's copies in flight land (a second wait of at
 * most the default) and ends the block; that evaluation's results are not
 * valid, and the context stays usable. With `unmet` nonzero every such wait
 * targets a barrier that nothing completes, so each runs out after `cycles`:
 * a test of that path without any fault. Synchronises the device and drops
 * the plan's cached graphs. */
sag_status sag_plan_set_wait_limit(sag_plan_t plan, int64_t cycles, int32_t unmet);

/* Waits for `stream`, then returns and clears the plan's latched device-side
 * status (SAG_OK, SAG_ENONFINITE or SAG_ETIMEOUT). When a block that gave up a
 * wait also ran out of time waiting for its own bulk copies in flight, the
 * status is SAG_ETIMEOUT with a message saying so: copies may then still have
 * landed in shared memory after the block ended, and the context should be
 * treated as suspect. */
sag_status sag_sync_status(sag_plan_t plan, void* stream);

/* Kernel timing, for profiling and roofline reporting. While enabled, every
 * kernel that sag_rhs / sag_rhs_parts / sag_rk2_step launch (not the graph
 * replays of sag_integrate) is bracketed by CUDA events recorded on the
 * launch stream. sag_profile_read waits for that work, adds each kernel's
 * total time (ms) and launch count to ms[id] and launches[id] for
 * id < min(n, SAG_NUM_KERNELS), and forgets the records. */
#define SAG_NUM_KERNELS 13
sag_status sag_profile_enable(sag_plan_t plan, int32_t on);
sag_status sag_profile_read(sag_plan_t plan, double* ms, int64_t* launches, int32_t n);
/* Name of kernel id (0 <= id < SAG_NUM_KERNELS), or NULL. */
const char* sag_kernel_name(int32_t id);

/* Algorithmic work of one launch of kernel id for this plan: *ops = arithmetic
 * instructions of the method (one FP32 add, multiply or FMA = 1 op for the
 * double-word path, one FP64 op for FP64 arithmetic; index arithmetic, loads
 * and stores excluded), *ops_fp64 = 1 if those are FP64 instructions, and
 * *bytes = the HBM bytes the step must move at minimum (its inputs and
 * outputs, not the workspace between kernels). Counts follow the radix
 * schedule and the double-word operation costs stated in the source. */
sag_status sag_kernel_work(sag_plan_t plan, int32_t id, double* ops, int32_t* ops_fp64,
                           double* bytes);

/* The method's own measure of one launch of kernel id, for roofline
 * reporting beside sag_kernel_work: *flops = nominal flops of the part of the
 * method the launch carries out (a real FFT of length L counted as
 * 2.5 L log2 L, split between the four-step column and row halves as
 * 2.5 L log2 M1 and 2.5 L log2 M2; a complex product 6, an add 2; inner
 * products 2 per factor element), whatever arithmetic carries it out; and
 * *workspace_bytes = the bytes of intermediate FFT workspace the launch writes
 * or reads beyond sag_kernel_work's algorithmic bytes (each transformed
 * vector's four-step intermediate, 16 bytes per complex value; each order's
 * spectral sum). Sec. 1 gives the method's cost as O(N D R log N). */
sag_status sag_kernel_method_work(sag_plan_t plan, int32_t id, double* flops, double* workspace_bytes);

/* JSON description of the plan's FFT geometry (per order: L, M1, M2, radix
 * schedules, block shapes), its launch layout, the split autotuner's
 * candidates, and launches_per_step: the kernel launches of one sag_integrate
 * step without diagnostics (the kernel nodes of the step captured as a graph,
 * not launched; -1 if the capture fails). Written to buf (NUL-terminated,
 * truncated to len). */
sag_status sag_plan_describe(sag_plan_t plan, char* buf, size_t len);

/* Loss term without allocation: q = sum_d Q^(d)[n] (same definition and
 * symmetrize_q meaning as sag_rhs_parts) for one CP system, computed directly
 * from caller-owned device buffers with no plan. The paper has no counterpart;
 * it exists for callers that cannot allocate device memory (code running under
 * an allocator it does not own, in a fixed-budget memory pool, or in a process
 * that reserved its device memory up front): this call performs no cudaMalloc,
 * cudaFree or other allocation.
 *   sys: fmt = SAG_CP, factors_on_device = 1, factors a device pointer in the
 *        layout of sag_system; rank is read on the host. As in sag_plan, a CP
 *        rank of 0 leaves an order out, and one order needs rank >= 1.
 *   n, q: device vectors of length N (may not alias).
 * Limits: V = sum_d d R_d <= 2048 and V * ceil(N / 8192) <= 32768; larger
 * systems, host pointers or TT kernels return SAG_EINVAL / SAG_EUNSUPPORTED
 * with a message. Partial sums and loss weights live in one static device
 * array of 288 KB that every device loading the library keeps until exit; all
 * calls share it, so calls that overlap on the GPU (any streams) race. The
 * first call on each device looks up that array's device address
 * (cudaGetSymbolAddress), so make it before any stream capture. Asynchronous
 * on `stream`. */
sag_status sag_loss_noalloc(const sag_system* sys, int32_t symmetrize_q, const double* n, double* q,
                            void* stream);

/* The parametric factors' generator on its own, for checking it: out[i-1] =
 * u i^a for i = 1..N (N <= 2^22, |a| <= 2.5), evaluated in double-word FP32
 * exactly as the forward FFT of a SAG_CP_POWER plan does and returned as the
 * FP64 sum of the two words. out is a device vector of N doubles. Allocates
 * its two small tables, waits for `stream` and frees them before returning. */
sag_status sag_power_eval(double u, double a, int32_t N, double* out, void* stream);

/* Releases the plan (after the work queued on it has finished). NULL is a no-op. */
void sag_plan_destroy(sag_plan_t plan);

/* Message of the last failing call on this host thread ("" if none). */
const char* sag_last_error(void);

/* Library version string. */
const char* sag_version(void);

#ifdef __cplusplus
}
#endif
#endif
