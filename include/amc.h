/*
 * amc.h - C ABI of the GB300 (sm_103a) quasi-Monte Carlo American option
 * pricer.
 *
 * Method (Cvetanoska & Stojanovski, "Using High Performance Computing and
 * Monte Carlo Simulation for Pricing American Options"):
 *   - the option is Bermudan on t_j = j*T/m, j = 1..m (§III.E, §V);
 *   - quasi-random points mapped to N(0,1) by an inverse cumulative normal
 *     (§III.D): here 32-bit Sobol' points (Joe-Kuo direction numbers,
 *     Gray-code order, point index = path index) with a digital XOR shift
 *     drawn from SplitMix64(seed);
 *   - Brownian-bridge path construction (ref. [13]): breadth-first bisection;
 *   - the GBM step of Eq. 9, evaluated in log space;
 *   - a backward early-exercise sweep: Longstaff-Schwartz regression
 *     (ref. [12]; §V backward induction) by default, or the paper's own
 *     pathwise rule (Eqs. 10-11), or no early exercise (Eqs. 6-8);
 *   - the price is the path average (Eq. 6) discounted to t = 0.
 *
 * Conventions for every entry point:
 *   - return 0 (AMC_OK) or a negative AMC_E* code; no exception crosses the
 *     ABI; amc_strerror() names a code;
 *   - host pointers are read or written only during the call; device
 *     pointers ("_dev") must stay valid until the work queued on the given
 *     stream has finished; a NULL stream means the legacy default stream;
 *   - the context owns all scratch memory; calls on one context are
 *     serialised by the caller, except amc_serve_*, which is thread-safe;
 *   - option validation: S0, K, sigma, T > 0 and finite, r finite,
 *     1 <= n_steps <= AMC_MAX_STEPS, 1 <= n_paths <= AMC_MAX_PATHS,
 *     basis in 1..4 (LSM rule), type in {AMC_PUT, AMC_CALL}; a bad option
 *     returns AMC_EINVAL before any device work.
 */
#ifndef AMC_H
#define AMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AMC_OK 0
#define AMC_EINVAL (-1)   /* bad argument                                   */
#define AMC_ENOMEM (-2)   /* context arena or device memory exhausted       */
#define AMC_ECUDA (-3)    /* a CUDA runtime call failed                     */
#define AMC_ETIMEOUT (-4) /* a device-side wait ran past its time limit     */
#define AMC_EBUSY (-5)    /* serving admission refused (memory or slots)    */
#define AMC_PENDING (-6)  /* serving request not finished yet               */
#define AMC_ENOTFOUND (-7)/* unknown serving ticket                         */
#define AMC_ECANCELED (-8)/* serving request cancelled before it ran        */

#define AMC_MAX_STEPS 512          /* direction-number table limit          */
#define AMC_MAX_PATHS (1LL << 31)  /* 32-bit Sobol' point index             */

enum { AMC_PUT = 0, AMC_CALL = 1 };
/* Exercise rules: Longstaff-Schwartz regression (ref. [12]); the paper's
 * pathwise rule, Eqs. 10-11 (an upper bound, §V); European, Eqs. 6-8.      */
enum { AMC_RULE_LSM = 0, AMC_RULE_PAPER_UB = 1, AMC_RULE_EUROPEAN = 2 };
/* Precision: all-FP64 paths, sums and solve; or FP32 paths with
 * compensated (double-float) FP32 sums, FP64 solve and FP64 final price.
 * AMC_MIXED stays within 2e-4 K of the FP64 estimate where the LSM
 * estimator is stable at FP32 precision.  Where a wide moneyness range
 * meets a rich basis (volatility 150 % with p = 4, a 10-year call at 40 %
 * with p = 4, a call with S0/K = 1.4, sigma 34 %, T = 1.7 and p = 3),
 * exercise decisions near the fitted boundary flip under perturbations of
 * order 1e-7 and the FP64 estimate itself moves by more than 2e-4 K under
 * FP32-level noise; price such options with AMC_FP64 (or a smaller basis).  */
/* AMC_MIXED16 is AMC_MIXED with the path array stored as the moneyness
 * y = S/K - 1 in IEEE binary16 (round to nearest even) instead of S in
 * FP32: half the bytes of S, and the sweeps read y as stored.  The
 * paths it stores are those of AMC_MIXED rounded to binary16 (a relative
 * step of 2^-11 in y).  Accepted by amc_generate_paths, amc_sweep and
 * amc_fit_boundary (the LSM rule, no Greeks), amc_price_american and
 * amc_price_device (LSM), and amc_price_batch and amc_price_batch_device
 * (every option LSM); AMC_EINVAL everywhere else.  The rounding moves the
 * estimate by far less than 2e-4 K on options where LSM is stable at FP32
 * precision (3e-5 K on the 252-date put); on the unstable kind above it
 * moves by up to several 1e-4 K.                                           */
enum { AMC_FP64 = 0, AMC_MIXED = 1, AMC_MIXED16 = 2 };

/* One option.  72 bytes, naturally aligned.                                */
typedef struct amc_option {
    double S0, K, r, sigma, T; /* spot, strike, rate, volatility, maturity  */
    int32_t n_steps;           /* m exercise dates t_j = j T / m            */
    int32_t basis;             /* LSM basis size p: {1, y, .., y^(p-1)}, y = S/K - 1
                                  (the span of {1, S, .., S^(p-1)})      */
    int64_t n_paths;           /* N Sobol' points / paths                   */
    int32_t type;              /* AMC_PUT or AMC_CALL                        */
    int32_t rule;              /* AMC_RULE_*                                 */
    uint64_t seed;             /* digital-shift seed                         */
} amc_option;

/* Result of one pricing.  price and std_err are at t = 0; std_err is the
 * sample standard deviation of the discounted path values over sqrt(N);
 * delta and vega are filled by the Greeks calls only; degenerate_dates
 * counts LSM dates with fewer than p in-the-money paths or a Cholesky
 * pivot <= 1e-12 after equilibration (no exercise there).                  */
typedef struct amc_result {
    double price, std_err, delta, vega;
    int32_t degenerate_dates;
    int32_t status;            /* AMC_OK or the error of this option        */
    float ms_gen, ms_sweep;    /* device time of path generation and sweep  */
} amc_result;

/* Device result block written by the asynchronous calls: 8 doubles,
 * [price, std_err, delta, vega, degenerate_dates, status, 0, 0].           */
#define AMC_RES_DOUBLES 8
/* Exercise boundary of one LSM option: AMC_COEF_STRIDE doubles per date
 * d = 1..m (row d-1): c_0..c_3, the continuation value divided by K as a
 * polynomial in the moneyness y = S/K - 1 (c_k = 0 for k >= basis), then a
 * degenerate flag (nonzero: no exercise at d; always set for d = m).       */
#define AMC_COEF_STRIDE 5

typedef struct amc_ctx amc_ctx;

/* ---------------------------------------------------------------- context */
/* Library and error strings.  No GPU needed.                               */
const char *amc_strerror(int code);
int amc_version(void);

/* Create a context on CUDA device `device` with a device arena of
 * `arena_bytes` (0 = 60% of the free device memory) for path storage and
 * scratch.  Uploads the direction-number table.  *out is set on success.  */
int amc_ctx_create(int device, size_t arena_bytes, amc_ctx **out);
int amc_ctx_destroy(amc_ctx *ctx);
/* Time limit of every device-side wait (default 2 s).                      */
int amc_ctx_set_timeout(amc_ctx *ctx, double seconds);
/* Host-side fault injection for tests (never traps or faults the GPU):
 *   kind 1: in the next LSM sweep, CTA 0 of the first job skips its arrival
 *           at exercise date `arg`, so the other CTAs' waits run out and the
 *           call returns AMC_ETIMEOUT;
 *   kind 2: the next arena reservation fails (AMC_ENOMEM);
 *   kind 3: the next LSM sweep runs the streaming sweep of large options
 *           (cash flows in device memory, one pass and one solve per date)
 *           whatever its path count, so that it can be tested on small
 *           options;
 *   kind 4: the next mixed-precision LSM launch of amc_price_batch,
 *           amc_greeks, their _device forms or the serving loop takes the
 *           launch tag `arg` (1 <= arg < 2^22) of its cross-CTA exchange
 *           units instead of a new one, so that units an earlier launch
 *           left in the same arena memory carry the tag the new launch
 *           waits for: a test that stale exchange data is never taken for
 *           fresh (results must not change);
 *   kind 0: clear.                                                          */
int amc_ctx_inject(amc_ctx *ctx, int kind, int64_t arg);
/* Opt-in device timing of the hot path's launches (off by default): with
 * profiling on, every path-generation launch and every sweep launch of
 * this context (single options, batches, Greeks, serving) is bracketed by
 * CUDA events on its stream, with its work in path-steps (the sum of
 * n_paths * n_steps over the options it covers); the waves of a batch then
 * run one after another on one stream, so that each launch's time is its
 * own rather than shared with an overlapping launch.  amc_ctx_profile waits for
 * the recorded launches, returns the summed device times (ms), launch
 * counts and path-steps of each kind since the previous call, and clears
 * them; any pointer may be null.                                           */
int amc_ctx_set_profiling(amc_ctx *ctx, int enable);
int amc_ctx_profile(amc_ctx *ctx, double *gen_ms, double *sweep_ms, int64_t *gen_launches,
                    int64_t *sweep_launches, int64_t *gen_path_steps, int64_t *sweep_path_steps);
/* Bytes of the arena currently free / total.                               */
int amc_ctx_memory(amc_ctx *ctx, size_t *free_bytes, size_t *total_bytes);

/* ------------------------------------------------- host-only helpers */
/* None of these touches a GPU.                                             */
int amc_validate_option(const amc_option *opt);
/* Row stride (elements) of the date-major path array S[m][ld]: n_paths
 * rounded up to a multiple of 32.                                          */
int64_t amc_path_ld(int64_t n_paths);
/* Bytes of S for one option: n_steps * ld * (8 for AMC_FP64, 4 for
 * AMC_MIXED, 2 for AMC_MIXED16).                                           */
size_t amc_path_bytes(int n_steps, int64_t n_paths, int prec);
/* Digital shifts: out[d] = high 32 bits of the d-th SplitMix64 output.     */
int amc_digital_shifts(uint64_t seed, int n_dims, uint32_t *out);
/* Sobol' direction numbers v_{b+1} of dims 0..n_dims-1: out[d*32 + b].    */
int amc_sobol_directions(int n_dims, uint32_t *out);
/* Bridge schedule in coordinate order k = 0..m-1: the date filled by
 * coordinate k and the dates it is conditioned on (0 = W(0) = 0).          */
int amc_bridge_schedule(int n_steps, int32_t *date, int32_t *left, int32_t *right);
/* The same bridge (ref. [13]; §III.D) in the depth-first order that path
 * generation evaluates it (inspection path; each array holds n_steps
 * entries): node k forms W(t_date[k]) = wl[k] W[sl[k]] + wr[k] W[sr[k]] +
 * sdu[k] sqrt(T / n_steps) z_coord[k] from the per-path stack W[0..n_slots-1],
 * which starts at 0, and stores it in W[so[k]].  W(0) = 0 takes no slot: a
 * node on [0, t_r] has wl = 0 and reads its right end point twice, and the
 * first node (t_m) has wl = wr = 0.  AMC_EINVAL for n_steps outside
 * 1..AMC_MAX_STEPS or a null pointer.                                      */
int amc_bridge_plan(int n_steps, int32_t *coord, int32_t *date, int32_t *sl, int32_t *sr, int32_t *so, double *wl,
                    double *wr, double *sdu, int32_t *n_slots);
/* CTAs the sweep gives one option of n_paths paths in precision `prec`
 * under `rule` (a pure function of these and the device's SM count), and
 * the paths each sweep thread owns.  AMC_EINVAL when the option's per-path
 * state does not fit on chip: the mixed LSM sweep holds up to
 * min(SMs, 160) * 7680 paths (1.17 M on 152 SMs), the other sweeps up to
 * SMs * 8192.                                                              */
int amc_plan_sweep(int64_t n_paths, int sm_count, int prec, int rule, int32_t *ctas, int32_t *paths_per_thread);

/* ------------------------------------ step-level calls (device buffers) */
/* Shifted Sobol' integers x[d][i], d < n_dims, i < n_points, row stride
 * ld >= n_points (test and inspection path; the pricer never stores them). */
int amc_sobol(amc_ctx *ctx, int n_dims, int64_t n_points, uint64_t seed,
              uint32_t *x_dev, int64_t ld, void *stream);
/* Steps 1-3: paths S[j-1][i] = S_i(t_j), date-major, row stride ld >=
 * amc_path_ld(n_paths) and a multiple of 32; S 16-byte aligned (else
 * AMC_EINVAL); float for AMC_MIXED, double for AMC_FP64, and for
 * AMC_MIXED16 the binary16 moneyness S_i(t_j)/K - 1 (uint16 bits).  Entries
 * n_paths <= i < ld of a row may receive the values of the extra Sobol'
 * points; nothing beyond ld is written.                                    */
int amc_generate_paths(amc_ctx *ctx, const amc_option *opt, int prec,
                       void *S_dev, int64_t ld, void *stream);
/* Steps 1-3 with the paper's randomisation of the points (§III.D) in place
 * of the digital shift: each dimension's array of quasi-random points is
 * permuted by a linear congruential generator.  Path i takes the unshifted
 * Sobol' point pi_d(i) in dimension d, pi_d(i) = L_d(i) applied again while
 * the value is >= n_paths, L_d(x) = (a_d x + c_d) mod M; M is the least
 * power of two >= n_paths, a_d = 1 mod 4 and c_d odd (full period, so pi_d
 * is a permutation of 0..n_paths-1); a_d and c_d come from outputs 2d and
 * 2d+1 of SplitMix64(opt->seed) (amc_lcg_params).  Storage, layout and
 * errors as amc_generate_paths; the sweeps take these paths unchanged.    */
int amc_generate_paths_permuted(amc_ctx *ctx, const amc_option *opt, int prec,
                                void *S_dev, int64_t ld, void *stream);
/* The permutation's parameters of dimensions 0..n_dims-1 for n_points
 * points: a[d] = 4 (r_2d mod max(M/4, 1)) + 1, c[d] = (r_2d+1 mod M) | 1,
 * *M the modulus.  No GPU.                                                 */
int amc_lcg_params(uint64_t seed, int n_dims, int64_t n_points, uint32_t *a, uint32_t *c, uint64_t *M);
/* Step 4 on caller paths S (as written by amc_generate_paths), result into
 * res_dev[AMC_RES_DOUBLES].  with_greeks != 0 also fills delta and vega
 * (frozen exercise boundary).  Asynchronous.  An LSM option with more paths
 * than the register-resident sweep holds (about 1.2 M on 152 SMs) runs the
 * streaming sweep: its cash flows in context memory, one pass and one solve
 * per date (16 bytes of traffic per path and date); the pathwise rules run
 * on a larger grid.  Greeks, batches and serving keep the register-resident
 * sizes (AMC_EINVAL beyond them).                                          */
int amc_sweep(amc_ctx *ctx, const amc_option *opt, int prec, const void *S_dev,
              int64_t ld, int with_greeks, double *res_dev, void *stream);
/* Steps 1-4 into caller storage: amc_generate_paths then amc_sweep.        */
int amc_price_device(amc_ctx *ctx, const amc_option *opt, int prec, void *S_dev,
                     int64_t ld, double *res_dev, void *stream);

/* Second Longstaff-Schwartz pass (ref. [12]; the paper values in sample,
 * with the paths it regresses on).  amc_fit_boundary runs the LSM sweep of
 * an AMC_RULE_LSM option on S (as amc_sweep, in-sample result into
 * res_dev) and also writes the fitted boundary into
 * coef_dev[n_steps * AMC_COEF_STRIDE].  amc_value_boundary values the paths
 * S with a given boundary and no regression: on each path CF = h(S_m), then
 * for d = m-1..1, CF <- CF e^{-r dt} and CF = h(S_d) if d is not degenerate,
 * S_d is in the money and h(S_d) > K c_d(y_d); price = e^{-r dt} mean CF
 * (result block as amc_sweep, delta and vega 0, degenerate_dates = flagged
 * dates).  With paths independent of those the boundary was fitted on, this
 * is a low-biased estimator of the Bermudan value; with the fitting paths
 * it repeats the in-sample exercise decisions.  One streaming read of S,
 * no reduction across the grid.  Both asynchronous; S, ld as amc_sweep;
 * coef_dev 8-byte aligned device memory (AMC_EINVAL otherwise, or if the
 * option's rule is not AMC_RULE_LSM).                                      */
int amc_fit_boundary(amc_ctx *ctx, const amc_option *opt, int prec, const void *S_dev,
                     int64_t ld, double *coef_dev, double *res_dev, void *stream);
int amc_value_boundary(amc_ctx *ctx, const amc_option *opt, int prec, const void *S_dev,
                       int64_t ld, const double *coef_dev, double *res_dev, void *stream);

/* Steps 1-4 with no path array: path generation values every path as its
 * dates are formed (the bridge forms them out of order) and stores nothing,
 * for the rules that need no regression across paths.  AMC_RULE_PAPER_UB:
 * Eqs. 10-11, whose backward recursion is the maximum over t_0..t_{m-1} of
 * the discounted payoffs, with the Black-Scholes value over the last
 * interval taken at t_{m-1}; AMC_RULE_EUROPEAN: Eqs. 6-8; AMC_RULE_LSM with
 * a fitted boundary coef_dev (as written by amc_fit_boundary): the
 * valuation of amc_value_boundary on the option's own points (paths of
 * opt->seed), which is the out-of-sample price when the boundary was fitted
 * on other points.  coef_dev must be null for the other rules.  Result
 * block as amc_sweep / amc_value_boundary.  Same points and decisions as
 * generating, storing and then sweeping the paths; the sums are taken in
 * another fixed order.  Asynchronous.                                      */
int amc_price_fused(amc_ctx *ctx, const amc_option *opt, int prec, const double *coef_dev, double *res_dev,
                    void *stream);

/* Dual upper bound of a fitted boundary (the dual formulation of §IV,
 * ref. [11], with the Andersen-Broadie martingale of the boundary).  On each
 * outer path i of S (an AMC_RULE_LSM option's paths, as amc_sweep) and for
 * each date t_j < T, n_inner inner paths start from S_j(i), move by the exact
 * GBM step of Eq. 9 and stop at the first later date where the boundary
 * coef_dev exercises (as amc_value_boundary; always at t_m); Q_j(i) is the
 * mean of their payoffs discounted to t_j.  With D_j = e^{-r t_j},
 * Z_j = D_j h(S_j), L_j = Z_j where the boundary exercises at t_j and D_j Q_j
 * elsewhere (L_m = Z_m), L0 = mean over i of L_1, and
 * M_j = sum_{l<=j} (L_l - D_{l-1} Q_{l-1}) with D_0 Q_0 = L0:
 * U(i) = max_{j=1..m} (Z_j - M_j).  res_dev = [mean U, std_err of U, 0, 0,
 * flagged dates, status, L0, inner steps simulated]; U_dev[n_paths]
 * (device, 8-byte aligned, may be null) receives U(i).  Inner path k
 * (0-based) from date j of outer path i (0-based) owns the H = ceil(m/2)
 * SplitMix64 outputs number
 * n = ((i m + j - 1) n_inner + k) H + q, q = 1..H, of inner_seed, that is
 * mix(inner_seed + n 0x9E3779B97F4A7C15); its steps 2q-1 and 2q (to dates
 * j + 2q - 1, j + 2q) take the normals Phi^-1((x + 1/2) 2^-32) of the high
 * and of the low 32 bits x of output q.  FP32 inner paths under
 * AMC_MIXED (FP64 sums), all FP64 under AMC_FP64.  AMC_EINVAL for a rule
 * other than AMC_RULE_LSM, n_inner < 1 or > AMC_DUAL_MAX_INNER,
 * n_paths > 2^31 - 1, misaligned pointers, or more than AMC_DUAL_MAX_WORK
 * possible inner steps (n_paths n_inner m (m-1) / 2).  Asynchronous.      */
#define AMC_DUAL_MAX_WORK (1LL << 40)
#define AMC_DUAL_MAX_INNER (1LL << 29)   /* two dates' inner paths index one 32-bit window */
int amc_dual_upper(amc_ctx *ctx, const amc_option *opt, int prec, const void *S_dev, int64_t ld,
                   const double *coef_dev, int64_t n_inner, uint64_t inner_seed, double *res_dev,
                   double *U_dev, void *stream);

/* --------------------------------------------------- host-level calls */
/* Price one option (paths in the context arena), blocking; out on host.
 * The paper's problem statement: one option valued on a large number of
 * quasi-random paths (§III.D), inputs S0, K, T, r, sigma (Eqs. 1-5, §V),
 * m exercise dates t_j = j T/m (§III.E, §V), the early-exercise rule by
 * backward induction (§V; LSM, ref. [12], or Eqs. 10-11) and the average
 * of Eq. 6 discounted to t = 0 (Eqs. 7-8).                                 */
int amc_price_american(amc_ctx *ctx, double S0, double K, double r, double sigma,
                       double T, int n_steps, int64_t n_paths, int basis, int type,
                       uint64_t seed, int rule, int prec, amc_result *out);
/* Price n options (the many-options setting that motivates the paper's GPU
 * design, §III.D and §VI); each option's result equals its
 * amc_price_american result bit for bit.  Options are grouped into
 * arena-sized waves; within a wave path generation runs as one launch and
 * the sweeps as one persistent launch, each option on its own CTA group.
 * Blocking; out[n] on host.                                                */
int amc_price_batch(amc_ctx *ctx, const amc_option *opts, int n, int prec,
                    amc_result *out);
/* amc_price_batch on a caller's stream with the results on the device: the
 * result block of option i (AMC_RES_DOUBLES doubles, [price, std_err, 0, 0,
 * degenerate_dates, status, 0, 0]) into res_dev[i * AMC_RES_DOUBLES]
 * (device memory, 8-byte aligned, caller-owned; n * AMC_RES_DOUBLES
 * doubles).  The work is ordered after everything already queued on
 * `stream` and later work on `stream` is ordered after it; the call returns
 * without waiting for the GPU.  Results equal amc_price_batch's bit for bit.
 * Validation errors (AMC_EINVAL) are returned before any device work; a
 * per-option failure (e.g. AMC_ETIMEOUT) is that option's status in
 * res_dev; on any other nonzero return the contents of res_dev are
 * unspecified.  The context's arena is in use until the work has finished:
 * the next call on the context is ordered after it on the GPU.            */
int amc_price_batch_device(amc_ctx *ctx, const amc_option *opts, int n, int prec,
                           double *res_dev, void *stream);
/* Out-of-sample LSM price (paths in the context arena), blocking: the
 * boundary is fitted on the points of opt->seed (in-sample result into
 * fit, may be null) and applied to the independent points of value_seed
 * (result into value).  The second Longstaff-Schwartz pass of ref. [12];
 * the paper prices in sample (§V).                                         */
int amc_price_oos(amc_ctx *ctx, const amc_option *opt, uint64_t value_seed, int prec,
                  amc_result *fit, amc_result *value);
/* Lower and upper bounds of the Bermudan value, blocking: the boundary is
 * fitted on the points of opt->seed (in-sample result into fit, may be
 * null); on n_outer independent paths of outer_seed it is applied
 * (amc_value_boundary, into lower, may be null) and its dual upper bound
 * taken with n_inner inner paths per outer path and date (amc_dual_upper,
 * into upper).  The dual formulation of §IV (ref. [11]), against the
 * paper's own upper-bound rule (Eqs. 10-11, §V).                           */
int amc_price_dual(amc_ctx *ctx, const amc_option *opt, uint64_t outer_seed, int64_t n_outer, int64_t n_inner,
                   uint64_t inner_seed, int prec, amc_result *fit, amc_result *lower, amc_result *upper);
/* Price, delta and vega of n options (frozen-boundary pathwise adjoint:
 * the stopping dates of each path held fixed and e^{-r t} h(S_t)
 * differentiated along the path, dS/dS0 = S/S0, dS/dsigma = S (W - sigma t)
 * for the exact GBM step of Eq. 9).  The paper computes no Greeks.
 * AMC_RULE_LSM or AMC_RULE_EUROPEAN; blocking; host arrays of n.          */
int amc_greeks(amc_ctx *ctx, const amc_option *opts, int n, int prec,
               double *price, double *delta, double *vega);
/* amc_greeks on a caller's stream with device inputs and outputs, so that
 * a framework's autograd can keep spot, volatility and results on the GPU.
 * S0_dev and sigma_dev (device, n doubles each, either may be null) replace
 * opts[i].S0 and opts[i].sigma (which are then not read); their values are
 * checked on the device: an option whose replaced spot or volatility is
 * not finite and positive gets NaN price, delta and vega and status
 * AMC_EINVAL, the others are unaffected.  price_dev, delta_dev, vega_dev
 * (device, n doubles each) receive the results in input order; res_dev
 * (device, n * AMC_RES_DOUBLES doubles, may be null) also the full result
 * blocks with each option's status.  All pointers 8-byte aligned.
 * Ordering, return codes and results as amc_price_batch_device; the
 * results equal amc_greeks's bit for bit.                                  */
int amc_greeks_device(amc_ctx *ctx, const amc_option *opts, int n, int prec,
                      const double *S0_dev, const double *sigma_dev,
                      double *price_dev, double *delta_dev, double *vega_dev,
                      double *res_dev, void *stream);

/* ------------------------------------------------------------ serving */
/* Continuous batching of pricing requests (the paper's many-options
 * motivation, §III.D).  While serving runs, the context belongs to its
 * scheduler thread: the other pricing calls on it return AMC_EBUSY.        */
typedef struct amc_serve_config {
    size_t slot_bytes;   /* device memory per slot (0: arena / slots)       */
    int32_t slots;       /* concurrent batches on the GPU, 1..8             */
    int32_t max_batch;   /* requests per batch, 1..4096                     */
    int32_t max_pending; /* queue bound; submits beyond it get AMC_EBUSY    */
    int32_t prec;        /* AMC_MIXED or AMC_FP64                           */
} amc_serve_config;

typedef struct amc_serve_stats {
    int64_t submitted, launched, completed, rejected, batches, pending, cancelled;
} amc_serve_stats;

/* Start the scheduler thread.  Admission is by memory footprint: a request
 * whose paths and scratch exceed one slot is refused at submit (AMC_EBUSY);
 * otherwise it waits until a slot with room is free.  The oldest pending
 * request fixes the launch group of the next batch.                        */
int amc_serve_start(amc_ctx *ctx, const amc_serve_config *cfg);
/* Queue one request (thread-safe, non-blocking); *ticket identifies it.    */
int amc_serve_submit(amc_ctx *ctx, const amc_option *opt, uint64_t *ticket);
/* AMC_PENDING until done; then the result and the latency from submit to
 * completion (seconds), and the ticket is released.  Thread-safe.          */
int amc_serve_poll(amc_ctx *ctx, uint64_t ticket, amc_result *out, double *latency_s);
/* Up to `cap` finished requests, released; *n_out of them.  Thread-safe.   */
int amc_serve_drain(amc_ctx *ctx, uint64_t *tickets, amc_result *out, double *latency_s, int cap,
                    int *n_out);
/* Cancel a request that is still queued: it leaves the queue and finishes
 * at once with status AMC_ECANCELED (poll / drain hand it out).  AMC_EBUSY
 * if it is already on the GPU or finished (it completes normally),
 * AMC_ENOTFOUND for an unknown or released ticket.  Thread-safe.           */
int amc_serve_cancel(amc_ctx *ctx, uint64_t ticket);
int amc_serve_stats_get(amc_ctx *ctx, amc_serve_stats *out);
/* Finish every queued request, then stop the scheduler.                    */
int amc_serve_stop(amc_ctx *ctx);

/* ------------------------------------------- allocation-free sweep */
/* Step 4 (as amc_sweep) without a context and without allocating device
 * memory.  The paper has no counterpart: this entry point exists for
 * callers that may not allocate, e.g. a host framework that owns the whole
 * device-memory budget and forbids libraries to grow it, or a latency-
 * critical loop that cannot take the device-wide synchronisation of
 * cudaMalloc/cudaFree, or a plugin hook that holds no amc_ctx (creating one
 * allocates).  The caller passes the paths S_dev (as written by
 * amc_generate_paths) and the result block res_dev[AMC_RES_DOUBLES].
 *   Sizes: only options that the register-resident sweeps hold are
 * accepted (amc_plan_sweep succeeds: a mixed LSM option up to
 * min(SMs, 160) * 7680 paths, 1.17 M on 152 SMs; an FP64 LSM or pathwise
 * option up to SMs * 8192 paths).  amc_sweep falls back to the streaming
 * sweep or an uncapped grid beyond those sizes; this call has no fallback
 * and returns AMC_EINVAL before any device work.
 *   Scratch: a file-scope device array of amc_sweep_noalloc_capacity()
 * bytes (16 MiB) that every GPU that runs this call holds until the process
 * exits.  An option needs 67,840 bytes plus its exchange data:
 * 88*(n_steps+2)*C bytes for the mixed LSM sweep, 96*n_steps*C bytes
 * otherwise, C = the CTA count of amc_plan_sweep (all accepted mixed LSM
 * options fit; an FP64 LSM option with 512 dates and 2^20 paths does not);
 * an option that needs more returns AMC_EINVAL before any device work.
 *   The first call on a device looks up the array's device address and the
 * SM count (no allocation).  With CUDA's lazy module loading (the default)
 * that lookup also loads the array, so the driver reserves its 16 MiB at
 * that first call: make it before any latency-critical loop and before any
 * stream capture.
 *   Every call on a device shares the array.  A call clears what must start
 * at zero (its counters and, for the mixed LSM sweep, the exchange units it
 * polls) on `stream` before its kernels run.  Calls whose work overlaps on
 * the GPU (other streams, or other host threads) race on the array and
 * must be serialised by the caller.  Every device-side wait gives up after
 * 2 s (status AMC_ETIMEOUT in res_dev).  Uses the current device; results
 * are bit-identical to amc_sweep's on the same paths.                      */
int amc_sweep_noalloc(const amc_option *opt, int prec, const void *S_dev, int64_t ld,
                      int with_greeks, double *res_dev, void *stream);
size_t amc_sweep_noalloc_capacity(void);

#ifdef __cplusplus
}
#endif
#endif /* AMC_H */
