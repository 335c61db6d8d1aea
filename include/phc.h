/*
 * phc.h -- C ABI of the GB300 path-tracking library.
 *
 * The library tracks the solution paths of polynomial homotopies on one
 * NVIDIA GB300 (sm_103a): the total-degree homotopy of a square system, the
 * top-dimensional embedded system of a numerical irreducible decomposition
 * and the cascade of homotopies down to dimension zero (Verschelde, "A
 * Blackbox Polynomial System Solver on Parallel Shared Memory Computers",
 * Sections 2 and 3).  Paths are independent (Section 1), so every path is
 * tracked by one GPU thread, and the paths still running when most threads
 * are idle finish in tail kernels that give each one a warp (with the same
 * arithmetic, so results do not depend on where a path finishes); all
 * compute runs in the library's CUDA kernels.
 *
 * Conventions
 *  - Every function returns PHC_OK (0) or a negative PHC_E* code; the message
 *    of the last failure on the calling thread is phc_last_error().
 *  - Complex numbers are phc_cd {re, im} (16 bytes, the layout of CUDA's
 *    double2 and of numpy/torch complex128).
 *  - "device" arrays live in the memory of the current CUDA device and are
 *    owned by the caller; the library reads and writes them on the stream
 *    passed as `cuda_stream` (a cudaStream_t; NULL is the legacy default
 *    stream).  Calls return after enqueueing work, except where noted.
 *  - "host" arrays are owned by the caller and read during the call only.
 *  - Endpoint arrays are structs of arrays: x[j * n_paths + p] is unknown j
 *    of path p ("SoA [n_var][n_paths]").
 *  - A per-path numerical failure is not an error: it is class PHC_FAILED.
 *  - A handle keeps per-call scratch (queue and hand-off counters, records):
 *    tracking calls on one handle must not overlap on the GPU (issue them on
 *    one stream, or order the streams); different handles are independent.
 *  - The library never exits, aborts or traps on the device; no C++
 *    exception leaves an entry point (a failed host allocation returns
 *    PHC_ENOMEM; the outputs of that call are then undefined).
 */
#ifndef PHC_H
#define PHC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } phc_cd;

/* Opaque, library-owned homotopy handle; free with phc_destroy_homotopy. */
typedef struct phc_homotopy phc_homotopy;

enum {
    PHC_OK = 0,
    PHC_EINVAL = -1,        /* invalid argument or system                 */
    PHC_ENOMEM = -2,        /* host or device allocation failed           */
    PHC_ECUDA = -3,         /* a CUDA call failed (message names it)      */
    PHC_ETIMEOUT = -4,      /* a bounded device wait ran out (reserved: no
                               kernel of this library waits on another, so
                               no call returns it)                        */
    PHC_EUNSUPPORTED = -5   /* size or option outside what is built       */
};

/* Endpoint classes (int8 codes).  The paper counts paths that diverge "at
 * infinity" and separates regular from singular solutions (Sections 3.1 and
 * 4); the thresholds are in phc_opts. */
enum { PHC_REGULAR = 0, PHC_SINGULAR = 1, PHC_AT_INFINITY = 2, PHC_FAILED = 3 };

/* Why tracking stopped (phc_path_stats.stop). */
enum { PHC_STOP_REACHED = 0, PHC_STOP_DIVERGED = 1, PHC_STOP_STEP_MIN = 2, PHC_STOP_BUDGET = 3,
       PHC_STOP_NONFINITE = 4, PHC_STOP_SKIPPED = 5 /* not a start of this stage (phc_cascade_from) */ };

/* Arithmetic of the tracker.  FP32_INTERIOR runs the predictor stages
 * (H_t, Jacobian, factorization, solve) in single precision and factors the
 * Jacobian of every Newton correction in single precision while the step
 * ends at t <= fp32_t_max; the residual of every Newton correction stays
 * double, and so does everything after t = fp32_t_max (the end game).  A
 * single precision factorization whose pivots spread by more than
 * fp32_pivot_ratio counts as failed; a failed single precision step is retried in double and the
 * rest of that path stays in double. */
enum { PHC_PREC_FP64 = 0, PHC_PREC_FP32_INTERIOR = 1 };

#define PHC_MAX_VARS 12    /* largest number of unknowns of a tracked system */

/* Tracking options.  The paper fixes none of these; the defaults
 * (phc_default_opts) are the readings the CPU oracle uses too.
 *   predictor   classical 4th-order Runge-Kutta on dx/dt = -H_x^{-1} H_t
 *   corrector   <= max_corr_iters Newton steps at t + h; converged when
 *               ||dx|| <= corr_tol (1 + ||x||); rejected when a correction
 *               fails to shrink by corr_contract or none converges
 *   step        clamped to land on t = 1; times `expand` (<= h_max) after
 *               expand_after accepted steps in a row; times `shrink` after
 *               a rejection; h < h_min, max_steps steps, or max_steps_decade
 *               steps without 1-t crossing a power of ten stall the path
 *   end         a path that reaches t = 1 gets <= end_iters Newton steps at
 *               t = 1 (stop at ||dx|| <= end_tol (1 + ||x||))
 *   classes     norms are max_j max(|Re x_j|, |Im x_j|).
 *               AT_INFINITY: ||x|| > diverge_norm after an accepted step
 *                 (a polyhedral path: diverge_norm x max(1, ||x(0)||), as
 *                 its binomial start solution may lie beyond it); or
 *                 an endpoint with ||x|| > endpoint_inf_norm; or stalled at
 *                 t >= end_zone with ||x|| grown by more than growth_inf per
 *                 decade of 1-t over its last (<= 4) decade checkpoints.
 *               FAILED: non-finite values, or stalled before end_zone.
 *               REGULAR: reached t = 1, cond <= cond_regular and relative
 *                 residual <= res_regular.
 *               SINGULAR: everything else (stalled near t = 1 or reached
 *                 t = 1 with a large condition number).
 *               cond is the root condition number
 *                 max_j sum_i |(J^-1)_ji|_1 (1 + scale_i) / (1 + ||x||),
 *                 J = H_x(x,1), scale_i = sum over the terms of equation i
 *                 of |c|_1 |x^a|_1, |z|_1 = |Re z| + |Im z|;
 *               relative residual = max_i |H_i(x,1)|_1 / (1 + scale_i).
 *   slack_tol   z is zero when |z| <= slack_tol (1 + ||x||). */
typedef struct {
    double h_init, h_max, h_min;
    int32_t expand_after;
    double expand, shrink;
    int32_t max_corr_iters;
    double corr_tol, corr_contract;
    int32_t max_steps;
    int32_t max_steps_decade;
    double diverge_norm, endpoint_inf_norm, end_zone, growth_inf;
    int32_t end_iters;
    double end_tol;
    double cond_regular, res_regular, slack_tol;
    int32_t precision;       /* PHC_PREC_*                                  */
    double fp32_t_max;       /* FP32_INTERIOR: single precision for t < this */
    double fp32_pivot_ratio; /* FP32_INTERIOR: largest pivot spread accepted */
    int32_t block_threads;   /* threads per block; 0 = chosen by the library */
    int32_t max_blocks;      /* grid size cap; 0 = one wave of resident blocks */
    double tail_drain;       /* every tracking call: once this fraction of the tracker's threads
                                has found no path left to claim, every path that starts a new step
                                moves to a tail kernel that gives each path a group of threads
                                (FP32_INTERIOR: only paths whose remaining steps are all double);
                                the arithmetic is the same, operation for operation, so the
                                results do not change.  0 = never. */
    int32_t tail_threads;    /* threads per path in that kernel: 8 (N <= 8), 16 or 32; 0 = 32 */
    int32_t compact;         /* phc_track_paths, phc_track_from and the cascade stages, N >= 4: once
                                no path is left to claim, every 8 units each block moves its running
                                paths to its lowest threads, so that warps without a path stop
                                issuing (the arithmetic of a path does not change).  1 (default) on,
                                0 off */
    int32_t group_paths;     /* phc_track_polyhedral, phc_solve_polyhedral: 1 a group of threads per
                                path (tail_threads of them; 0: 32 for up to 7 unknowns, else 16), -1
                                one thread per path, 0 (default) a group per path unless the call's
                                paths exceed 32 waves of the groups resident on the GPU at once (the
                                same results either way) */
} phc_opts;

/* Per-path statistics (device array of these, optional). */
typedef struct {
    double t;        /* last t reached                                     */
    double h;        /* last step size                                     */
    double cond;     /* root condition number at the endpoint (see opts)   */
    double relres;   /* relative residual at t = 1                         */
    double norm_x;   /* max-norm of the endpoint                           */
    double growth;   /* log10 growth of ||x|| per decade of 1-t, last checkpoints */
    int32_t n_accept, n_reject;   /* accepted / rejected steps            */
    int32_t n_newton;             /* Newton corrections (tracking + end)  */
    int32_t n_solve;              /* evaluate + factor + solve units      */
    int32_t stop;                 /* PHC_STOP_*                           */
    int32_t n_fp32;               /* evaluate + solve units in single precision */
    int32_t grew;                 /* 1 when the growth test flagged the path */
    int32_t system;               /* system of the path in a batch handle  */
} phc_path_stats;

/* Host-side system lists, library-allocated (phc_embed); free with
 * phc_free_lists.  Equation i owns terms_per_eq[i] consecutive terms; term t
 * is coefs[t] * prod_j x_j^exps[t * n_var + j]. */
typedef struct {
    int32_t n_eq, n_var, n_terms;
    int32_t *terms_per_eq;   /* [n_eq]            */
    uint8_t *exps;           /* [n_terms][n_var]  */
    phc_cd *coefs;           /* [n_terms]         */
} phc_system_lists;

/* Fill *opts with the defaults described above.  Never fails for non-NULL. */
int phc_default_opts(phc_opts *opts);

/* Build the total-degree homotopy H(x,t) = (1-t) gamma g(x) + t f(x) of a
 * square system f (n_eq == n_var), g_i(x) = x_i^{d_i} - 1 with d_i the
 * total degree of equation i (the Bezout start system; Section 5 quotes the
 * Bezout bound).  The lists are host arrays: terms_per_eq [n_eq] (>= 1
 * each), exps [T][n_var] row-major (T = sum terms_per_eq), coefs [T].
 * The library copies them, compiles the evaluation tables and uploads them
 * to the current device; the handle owns that memory.
 * Errors: PHC_EINVAL for a non-square system, n_var outside
 * 1..PHC_MAX_VARS, an equation without terms or of degree 0, a non-finite
 * coefficient, or gamma of zero modulus; PHC_ENOMEM / PHC_ECUDA. */
int phc_make_homotopy(int n_eq, int n_var, const int32_t *terms_per_eq, const uint8_t *exps,
                      const phc_cd *coefs, phc_cd gamma, phc_homotopy **out);

/* A batch of n_systems total-degree homotopies that share the supports of
 * one square system (terms_per_eq, exps as in phc_make_homotopy) and differ
 * in their coefficients coefs [n_systems][T] and constants gammas
 * [n_systems] (host arrays): the same problem solved for many coefficient
 * values, e.g. a system and copies of it with random coefficients.  Path
 * p of system s has the global index s * prod d_i + p, so one
 * phc_track_paths call tracks every system in one launch; the stats record
 * of a path names its system.  Errors as phc_make_homotopy. */
int phc_make_homotopy_batch(int n_eq, int n_var, const int32_t *terms_per_eq, const uint8_t *exps, int n_systems,
                            const phc_cd *coefs, const phc_cd *gammas, phc_homotopy **out);

/* Paths that the last tracking call on h (phc_track_paths, phc_cascade_stage,
 * phc_cascade_from, phc_track_pipeline) moved to a tail kernel (opts.tail_drain),
 * and the evaluate+solve units those paths ran there (units_out may be
 * NULL); 0 when no such call ran or the option was 0.  Host call: waits for
 * cuda_stream (the stream of that call) before reading the device counters.
 * Errors: PHC_EINVAL for a NULL handle or paths_out; PHC_ECUDA. */
int phc_tail_paths(const phc_homotopy *h, void *cuda_stream, int64_t *paths_out, int64_t *units_out);

/* Number of paths of the total-degree homotopy, prod d_i (host call); for a
 * batch handle, n_systems * prod d_i. */
int phc_num_paths(const phc_homotopy *h, int64_t *out);

/* Track paths first_path .. first_path + n_paths - 1 of the total-degree
 * homotopy (path p starts at the roots of unity selected by the digits of p
 * in the mixed radix (d_1, ..., d_n), x_1 fastest) from t = 0 to t = 1 and
 * classify the endpoints.  opts may be NULL (defaults).
 * Outputs (device, caller-owned): x_out SoA [n_var][n_paths] phc_cd,
 * cls_out [n_paths] int8 (PHC_REGULAR ...), stats_out [n_paths] or NULL.
 * A call with sizes and options that an earlier call on h already had
 * allocates nothing and does not synchronise with the host (stream-ordered
 * memsets and kernel launches only), so it can be captured in a CUDA graph.
 * Errors: PHC_EINVAL for a NULL handle or output, a range outside
 * [0, num_paths), or invalid options; PHC_ECUDA. */
int phc_track_paths(phc_homotopy *h, int64_t first_path, int64_t n_paths, const phc_opts *opts, phc_cd *x_out,
                    int8_t *cls_out, phc_path_stats *stats_out, void *cuda_stream);

/* phc_track_paths in complex double double arithmetic (Section 5 and
 * Table 2: the solver run in double double, "quality up").  The same
 * readings as phc_track_paths (RK4 predictor, Newton corrector, step
 * control, tolerances, stall and divergence rules), but the point, the
 * Runge-Kutta stages, H, H_x, H_t, the LU and the solves are complex double
 * double (t, step sizes and norms stay double, norms from the double parts);
 * the end Newton at t = 1 stops at ||dx|| <= 1e-26 (1 + ||x||), so a
 * regular endpoint is accurate to about 1e-30.  The endpoint is classified
 * from its double part as a double endpoint.  A unit costs about 15 times a
 * double precision one; there is no tail hand-off and no compaction
 * (opts.tail_drain, tail_threads, compact and precision are ignored).
 * Outputs (device, caller-owned): x_hi and x_lo SoA [n_var][n_paths] (the
 * endpoint is x_hi + x_lo), cls_out [n_paths], stats_out [n_paths] or NULL.
 * Errors: as phc_track_paths. */
int phc_track_paths_dd(phc_homotopy *h, int64_t first_path, int64_t n_paths, const phc_opts *opts, phc_cd *x_hi,
                       phc_cd *x_lo, int8_t *cls_out, phc_path_stats *stats_out, void *cuda_stream);

/* Track paths first_path .. first_path+n_paths-1 of a total-degree handle in
 * complex quad double (Section 5 and Table 2 run the solver in quad double;
 * its arithmetic is [HLB00]'s): the readings of phc_track_paths with the
 * point, the predictor stages, H, H_x, H_t, the LU and the solves in quad
 * double (t, step sizes and norms in double, from the leading parts); the end
 * Newton at t = 1 stops at ||dx|| <= 1e-58 (1 + ||x||).  x_out: device SoA
 * [4][n_var][n_paths], part k of coordinate j of entry q at
 * x_out[(k * n_var + j) * n_paths + q], the parts of decreasing magnitude and
 * their sum the endpoint; cls_out and stats_out as phc_track_paths (the
 * class from the leading parts).  One thread per path, its arrays in local
 * memory; no tail hand-off.  Errors: as phc_track_paths_dd. */
int phc_track_paths_qd(phc_homotopy *h, int64_t first_path, int64_t n_paths, const phc_opts *opts, phc_cd *x_out,
                       int8_t *cls_out, phc_path_stats *stats_out, void *cuda_stream);

/* The Cauchy endgame for singular endpoints (the paper distinguishes
 * isolated multiple solutions from regular ones, Section 4; Example 4.1's
 * point (2, 0) has multiplicity two).  A path converging to a singular
 * endpoint x* has near t = 1 an expansion x(s) = x* + sum_k a_k s^{k/c} in
 * s = 1 - t, c its cycle number; double precision Newton steps at t = 1
 * leave x* accurate to about 1e-8 only.  For each total-degree path
 * first_path .. first_path + n_paths - 1 the call tracks the path to
 * t = 0.99 (the tracker's predictor, corrector and step control; the step
 * clamped to land on 0.99), then around the circle 1 - t = 0.01 e^{i theta}
 * in complex t, sampling x at 16 angles per loop, until the path closes
 * (||x - x_start|| <= 1e-8 (1 + ||x_start||)) after c <= 8 loops.  The
 * estimate is the mean of the 16 c samples (Cauchy's integral formula in
 * s^{1/c}); it counts when its relative residual
 * max_i |H_i(x, 1)|_1 / (1 + scale_i) is <= 1e-10 (a path that runs to
 * infinity also closes, around a pole, and is rejected here).
 * Outputs (device): x_out SoA [n_var][n_paths] (the estimate, or the last
 * point when there is none), cycle_out [n_paths] int32 (c, 0 when there is
 * no estimate), stats_out [n_paths] or NULL (steps, Newton steps, relres of
 * the estimate, stop as phc_track_paths for a path that stopped before 0.99
 * or failed on the circle).  Total-degree and batch handles.
 * Errors: as phc_track_paths. */
int phc_endgame(phc_homotopy *h, int64_t first_path, int64_t n_paths, const phc_opts *opts, phc_cd *x_out,
                int32_t *cycle_out, phc_path_stats *stats_out, void *cuda_stream);

/* The embedded system E_D of Section 2.1 (eq. (2) for D = 1): unknowns
 * x_1..x_n, z_1..z_D; equation i is f_i(x) + sum_k gammas[i][k] z_k; equation
 * n_eq + k is hyper[k][0] + sum_j hyper[k][j+1] x_j + z_k.  A square f only
 * (square a non-square system first with phc_square).  gammas [n_eq][D] and
 * hyper [D][n_var + 1] are host arrays; when NULL they are drawn from
 * `seed` (standard complex Gaussian from a 64-bit linear congruential
 * generator with an xor-shift output: state s = seed ^ 0x9E3779B97F4A7C15,
 * advance s = s * 6364136223846793005 + 1442695040888963407, output the top
 * 53 bits of s ^ (s >> 29) as a uniform u in [0,1); two uniforms u1, u2 give
 * sqrt(-log u1) (cos 2 pi u2 + i sin 2 pi u2), so E|z|^2 = 1).  Host
 * call; *out is library-allocated (phc_free_lists).
 * Errors: PHC_EINVAL for a non-square f, top_dim < 0, or n_var + top_dim
 * above PHC_MAX_VARS; PHC_ENOMEM. */
int phc_embed(int n_eq, int n_var, const int32_t *terms_per_eq, const uint8_t *exps, const phc_cd *coefs,
              int top_dim, const phc_cd *gammas, const phc_cd *hyper, uint64_t seed, phc_system_lists **out);

/* A square system from a non-square one (Section 2.1): an underdetermined f
 * (n_eq < n_var) gains n_var - n_eq random hyperplanes
 * consts[k][0] + sum_j consts[k][j+1] x_j = 0 (consts [n_var - n_eq][n_var + 1]);
 * an overdetermined f (n_eq > n_var) gains n_eq - n_var new unknowns s_k
 * (after x), and equation i gains sum_k consts[i][k] s_k
 * (consts [n_eq][n_eq - n_var]).  A square f is returned unchanged.  consts
 * is a host array or NULL (then drawn from seed as in phc_embed).  The
 * result is square with max(n_eq, n_var) unknowns (at most PHC_MAX_VARS);
 * embed it with phc_embed.  Host call; *out is library-allocated
 * (phc_free_lists).  Errors: PHC_EINVAL for invalid lists or a square
 * system above PHC_MAX_VARS unknowns; PHC_ENOMEM. */
int phc_square(int n_eq, int n_var, const int32_t *terms_per_eq, const uint8_t *exps, const phc_cd *coefs,
               const phc_cd *consts, uint64_t seed, phc_system_lists **out);

/* One stage of the cascade of homotopies (Section 3.1, Figure 3): embedded_k
 * is a handle made from E_k (k >= 1 slacks, as phc_embed lays it out: z_k is
 * the last unknown and hyperplane k the last equation).  The homotopy keeps
 * every equation of E_k except hyperplane k, which becomes
 * (1-t) (hyper[k][0] + sum_j hyper[k][j+1] x_j) + z_k; at t = 1, z_k = 0 and
 * the remaining equations are E_{k-1}.  starts: device SoA
 * [n_var(E_k)][n_starts], solutions of E_k with z_k != 0.
 * Outputs (device): x_out SoA [n_var(E_k) - 1][n_starts] (z_k dropped),
 * cls_out [n_starts], slack_zero_out [n_starts] (1 when k > 1 and z_{k-1}
 * is zero, i.e. a candidate generic point of a (k-1)-dimensional set),
 * stats_out [n_starts] or NULL.
 * Errors: PHC_EINVAL (k < 1, k >= n_var, NULL arrays), PHC_ECUDA. */
int phc_cascade_stage(const phc_homotopy *embedded_k, int k, const phc_cd *starts, int64_t n_starts,
                      const phc_opts *opts, phc_cd *x_out, int8_t *cls_out, uint8_t *slack_zero_out,
                      phc_path_stats *stats_out, void *cuda_stream);

/* phc_cascade_stage fed directly by the previous stage's device outputs:
 * x_prev SoA [n_var(E_k)][n] with cls_prev [n] and slack_zero_prev [n] (the
 * outputs of phc_track_paths / phc_cascade_stage / phc_track_pipeline for
 * E_k); the stage tracks exactly the entries that start the next stage in
 * Section 3.1 -- regular endpoints whose slack z_k is not zero (cls_prev ==
 * PHC_REGULAR and slack_zero_prev == 0; slack_zero_prev NULL tests
 * |z_k| <= slack_tol (1 + ||x||) on x_prev) -- without compacting them, so a
 * chain of stages runs on one stream with no host round trip.  Outputs are
 * indexed like the inputs: x_out SoA [n_var(E_k) - 1][n], cls_out [n] (-1
 * for entries that were not starts), slack_zero_out [n], stats_out [n] or
 * NULL (stop = PHC_STOP_SKIPPED for entries that were not starts).
 * Errors: as phc_cascade_stage. */
int phc_cascade_from(const phc_homotopy *embedded_k, int k, const phc_cd *x_prev, const int8_t *cls_prev,
                     const uint8_t *slack_zero_prev, int64_t n, const phc_opts *opts, phc_cd *x_out, int8_t *cls_out,
                     uint8_t *slack_zero_out, phc_path_stats *stats_out, void *cuda_stream);

/* Track every path of n_h homotopies of different systems together (the
 * batching of many small problems: the paper's work crew over the paths of
 * many systems, Section 1).  Systems with the same number of unknowns share
 * one launch: each warp works on one system at a time with that system's
 * tables in its own shared memory, its lanes refill from the system's path
 * queue, and a warp whose lanes are all idle moves on to a system with
 * unclaimed paths; once every path is claimed, paths still running move
 * to a tail kernel (one warp per path, opts.tail_drain).  hs: host array
 * of n_h single-system handles; x_out, cls_out, stats_out: host arrays of
 * n_h device pointers, each as the
 * corresponding argument of phc_track_paths for that handle (stats_out or
 * any of its entries may be NULL).  The results equal n_h phc_track_paths
 * calls.  Errors: PHC_EINVAL for NULL or batch handles and NULL outputs,
 * PHC_ENOMEM, PHC_ECUDA. */
int phc_track_many(phc_homotopy *const *hs, int n_h, const phc_opts *opts, phc_cd *const *x_out,
                   int8_t *const *cls_out, phc_path_stats *const *stats_out, void *cuda_stream);

/* Coefficient-parameter homotopy H(x,t) = (1-t) gamma g(x) + t f(x)
 * (Section 2.3: the solutions of a random coefficient system are the start
 * solutions of the homotopy to the target system): g and f share the
 * supports terms_per_eq, exps (as in phc_make_homotopy); g has the
 * coefficients coefs_start [T], and there are n_systems targets
 * coefs_target [n_systems][T] (host arrays), e.g. one target per test
 * point of a membership test (phc_membership_test).  The handle has no
 * total-degree start system: phc_num_paths reports 0 and paths start from
 * caller-given solutions of g (phc_track_from).  Endpoints are classified
 * and refined (phc_refine_endpoints) with the exact target coefficients.
 * Errors: as phc_make_homotopy (the target lists are validated). */
int phc_make_parameter_homotopy(int n_eq, int n_var, const int32_t *terms_per_eq, const uint8_t *exps,
                                int n_systems, const phc_cd *coefs_start, const phc_cd *coefs_target,
                                phc_cd gamma, phc_homotopy **out);

/* Track n_starts paths of h from explicit points at t = 0 to t = 1 and
 * classify the endpoints.  starts: device SoA [n_var][n_starts], solutions
 * of the homotopy at t = 0 (of g for a parameter homotopy, of gamma
 * (x_i^{d_i} - 1) for a total-degree handle).  Entry q belongs to system
 * q / starts_per_system of a batch or parameter handle (starts_per_system
 * 0: every entry to system 0).  Outputs as phc_track_paths, indexed by
 * entry: x_out SoA [n_var][n_starts], cls_out [n_starts], stats_out or NULL.
 * Errors: PHC_EINVAL for NULL arrays, negative sizes or entries beyond the
 * handle's systems; PHC_ECUDA. */
int phc_track_from(phc_homotopy *h, const phc_cd *starts, int64_t n_starts, int64_t starts_per_system,
                   const phc_opts *opts, phc_cd *x_out, int8_t *cls_out, phc_path_stats *stats_out,
                   void *cuda_stream);

/* Homotopy membership test (Section 4.1, Example 4.1): does a point lie on
 * a k-dimensional solution set given by witness points?  The embedded
 * system E_k (host lists as phc_embed lays them out: unknowns x_1..x_n,
 * z_1..z_k; the last k equations are the hyperplanes, each with one
 * constant term, linear terms and its slack) has the m witness points
 * (device SoA [n_var][m]: solutions with every slack zero, the generic
 * points of the set).  For each test point z_t (host [p][n_var - k], the
 * x-coordinates), the constant c_j0 of hyperplane j moves to
 * c_j3 = -sum_i c_ji z_t,i, so that (z_t, 0) satisfies every hyperplane:
 * the homotopy (1-t) E_k(c_0) + t E_k(c_3) carries the witness points to
 * the generic points of the set on the moved hyperplanes; z_t lies on the
 * set when one of the m endpoints (regular or singular) equals (z_t, 0)
 * within tol (1 + ||z_t||) in every unknown.  p x m paths in one launch.
 * Outputs (device): on_out [p] (1 on the set, 0 not), and, unless NULL,
 * the endpoints x_out SoA [n_var][p * m] and their classes cls_out
 * [p * m] (test point t owns entries t*m .. t*m + m - 1).  The call
 * allocates its temporaries and returns after the work on cuda_stream has
 * finished.
 * Errors: PHC_EINVAL for k outside 1..n_var-1, m < 1, hyperplane rows of
 * another form, non-finite points, tol <= 0; PHC_ENOMEM; PHC_ECUDA. */
int phc_membership_test(int n_eq, int n_var, const int32_t *terms_per_eq, const uint8_t *exps,
                        const phc_cd *coefs, int k, const phc_cd *witness, int64_t m, const phc_cd *points,
                        int64_t p, double tol, const phc_opts *opts, uint8_t *on_out, phc_cd *x_out,
                        int8_t *cls_out, void *cuda_stream);

/* A prepared phc_track_many call (the same systems, options and output
 * arrays every time): phc_many_plan_create checks the arguments, groups the
 * systems by number of unknowns, uploads the per-system descriptors and
 * allocates the path counters, the hand-off records of the tail kernel and,
 * for handles given no stats array, per-path records of its own (host call:
 * it synchronises with the device; the helper streams it creates inherit
 * cuda_stream's priority).  phc_many_plan_run then enqueues, on cuda_stream,
 * only memsets and kernel launches -- no allocation, no host
 * synchronisation -- so it can be captured in a CUDA graph and replayed;
 * every run writes the outputs phc_track_many would.  Runs of one plan must
 * not overlap on the GPU, and the handles must outlive the plan.
 * phc_many_plan_destroy frees the plan after its work has finished.
 * Errors: as phc_track_many. */
typedef struct phc_many_plan phc_many_plan;
int phc_many_plan_create(phc_homotopy *const *hs, int n_h, const phc_opts *opts, phc_cd *const *x_out,
                         int8_t *const *cls_out, phc_path_stats *const *stats_out, void *cuda_stream,
                         phc_many_plan **out);
int phc_many_plan_run(phc_many_plan *plan, void *cuda_stream);
void phc_many_plan_destroy(phc_many_plan *plan);

/* The top stage and the cascade stage below it in one launch (Section 3.1,
 * Figure 3; the GPU counterpart of the paper's pipelining, Section 2.2).
 * Tracks paths first_path .. first_path + n_paths - 1 of the total-degree
 * homotopy of E_k (embedded_k as for phc_cascade_stage), classifies every
 * endpoint as its path ends and, when it is regular with z_k != 0
 * (|z_k| > slack_tol (1 + ||x||)), continues the same GPU thread on the
 * cascade homotopy E_k -> E_{k-1} from it, so stage k-1 starts while stage
 * k is still running and no host round trip separates them; paths still
 * running when most threads are idle finish, in either stage, in a tail
 * kernel (opts.tail_drain) that continues them the same way.
 * Outputs (device, caller-owned): the top stage as phc_track_paths (x_top
 * SoA [n_var][n_paths], cls_top [n_paths], stats_top or NULL) and, per top
 * path, the stage below: x_next SoA [n_var - 1][n_paths], cls_next (-1 where
 * the top endpoint was not continued), slack_zero_next (as
 * phc_cascade_stage), stats_next or NULL.  Top endpoints that only double
 * double refinement makes regular are not continued: refine the top stage
 * afterwards and pass those to phc_cascade_stage.
 * Errors: as phc_track_paths and phc_cascade_stage. */
int phc_track_pipeline(phc_homotopy *embedded_k, int k, int64_t first_path, int64_t n_paths, const phc_opts *opts,
                       phc_cd *x_top, int8_t *cls_top, phc_path_stats *stats_top, phc_cd *x_next, int8_t *cls_next,
                       uint8_t *slack_zero_next, phc_path_stats *stats_next, void *cuda_stream);

/* Refine endpoints of h (evaluated at t = 1) by Newton's method in complex
 * double double arithmetic (the paper's double double path, Section 5,
 * after Hida, Li and Bailey): every endpoint that reached t = 1
 * (stats[p].stop == PHC_STOP_REACHED), has class PHC_SINGULAR or
 * PHC_REGULAR and cond > cond_threshold gets <= max_iters iterations; it
 * becomes PHC_REGULAR when a correction falls to 1e-20 (1 + ||x||) and the
 * condition number at the refined point is <= cond_max, else PHC_SINGULAR.
 * Device arrays: x_hi_io SoA [n_var][n] (in/out, the double part),
 * x_lo_out SoA [n_var][n] (the low part; zero where untouched), cls_io [n],
 * stats_io [n] (cond updated).  For a cascade stage pass the handle of
 * E_{k-1} and the stage's outputs.
 * Errors: PHC_EINVAL, PHC_ECUDA. */
int phc_refine_endpoints(const phc_homotopy *h, phc_cd *x_hi_io, phc_cd *x_lo_out, int64_t n,
                         double cond_threshold, double cond_max, int max_iters, int8_t *cls_io,
                         phc_path_stats *stats_io, void *cuda_stream);

/* Largest n_paths phc_track_paths_noalloc accepts with stats_out == NULL. */
#define PHC_NOALLOC_MAX_PATHS 52428
/* Most paths phc_track_paths_noalloc moves to the tail kernel in one call. */
#define PHC_NOALLOC_MAX_HANDOFF 4096

/* phc_track_paths without any device allocation during the call (the paper
 * has no counterpart; this is a service to callers that cannot allocate).
 * Same arguments, outputs and errors as phc_track_paths, and the same
 * results.  Callers whose device memory belongs to another allocator (a
 * framework's caching allocator that reserved the free memory up front) or
 * that must not enter the allocator after start-up (latency-critical serving
 * loops) use it.  Its scratch -- the path-queue and hand-off counters, the
 * hand-off records of the tail kernel and, when stats_out is NULL, the
 * per-path records -- is one static device array of about 5.5 MiB
 * (256 B + 320 B * PHC_NOALLOC_MAX_HANDOFF + 80 B * PHC_NOALLOC_MAX_PATHS)
 * that every GPU loading the library holds until exit.  The first call on a
 * device (with that device current) looks up the array's address; make it
 * before any stream capture.  All calls share the array and it keeps the
 * last call's contents (the counters are cleared at each call): calls that
 * overlap on the GPU race, so serialise them.  With stats_out == NULL,
 * n_paths above PHC_NOALLOC_MAX_PATHS is rejected with PHC_EUNSUPPORTED.
 * The tail hand-off (opts.tail_drain) holds at most PHC_NOALLOC_MAX_HANDOFF
 * paths, so on launches of more threads it starts once no more than that
 * many threads still hold a path (a later start than tail_drain alone, the
 * same results), and opts.compact is ignored (no compaction).  The call resets the handle's hand-off counters:
 * phc_tail_paths reports 0 after it. */
int phc_track_paths_noalloc(phc_homotopy *h, int64_t first_path, int64_t n_paths, const phc_opts *opts,
                            phc_cd *x_out, int8_t *cls_out, phc_path_stats *stats_out, void *cuda_stream);

/* ---------------------------------------------------------------- measurement */

/* The FP64 rate of the current device, measured (the paper has no
 * counterpart: the trackers are bound by double precision arithmetic, and
 * this measures the peak their roofline divides by).  Launches 2 blocks per
 * SM of warps_per_block warps (1..32) on the stream; every thread runs 8
 * independent fused multiply-add chains for iters (1..1e8) iterations.
 * Synchronizes on the stream, then writes 2 x 8 x iters x threads / seconds
 * / 1e12 to *tflops_out (host).  Errors: PHC_EINVAL for NULL tflops_out or a
 * count out of range; PHC_ECUDA. */
int phc_fp64_probe(int warps_per_block, int64_t iters, double *tflops_out, void *cuda_stream);

/* ---------------------------------------------------------------- polyhedral homotopies */

/* Fine mixed cells of the Newton polytopes of a square system under an
 * integer lifting (Section 2.2: polyhedral homotopies solve a random
 * coefficient start system, one binomial start system per mixed cell, a cell
 * of volume V starting V paths; Figure 2 pipelines the making of the cells
 * with the tracking).  Host call, no device work.  Supports: the exponents
 * of each equation's terms (terms_per_eq [n], exps [T][n] as in
 * phc_make_homotopy; an equation may not list a monomial twice).
 * lift [T]: one integer per term in 0..2^20 (random values put the lifting
 * in general position).  A fine mixed cell picks two terms a_i < b_i
 * (global term indices) of every equation i such that some v in Q^n makes
 * <exps[a], v> + lift[a] equal on the pair and larger on every other term
 * of equation i; its volume is |det D|, D the n x n matrix with rows
 * exps[b_i] - exps[a_i].  The mixed volume (the sum of the volumes) counts
 * the isolated roots in (C*)^n of a system with these supports and
 * coefficients in general position (Bernstein).
 * The search runs on the host's threads (PHC_HOST_THREADS in the
 * environment, 1..64, sets their number; the cells and their order do not
 * depend on it).
 * Outputs: *n_cells_out (every cell) and *mixed_volume_out (may be NULL);
 * the first min(n_cells, max_cells) cells to cells_out [max_cells][n][2]
 * (a_i, b_i per equation) and their volumes to volumes_out [max_cells] (may
 * be NULL), in the order found (max_cells = 0 counts only).
 * Errors: PHC_EINVAL for n outside 1..PHC_MAX_VARS, NULL lists, an equation
 * without terms or with a repeated monomial, lifting values outside
 * 0..2^20, or a lifting not in general position (a third term on a cell's
 * lower facet: draw another lifting); PHC_EUNSUPPORTED when the exact
 * arithmetic would overflow 128 bits. */
int phc_mixed_cells(int n, const int32_t *terms_per_eq, const uint8_t *exps, const int32_t *lift,
                    int64_t max_cells, int32_t *cells_out, int64_t *volumes_out, int64_t *n_cells_out,
                    int64_t *mixed_volume_out);

/* The polyhedral homotopies of a system g with coefficients in general
 * position (host lists terms_per_eq, exps, coefs as in phc_make_homotopy)
 * over cells of phc_mixed_cells (host cells [n_cells][n][2], the same
 * lift [T]).  Cell k substitutes x = t^{v_k} y and divides equation i by
 * t^{beta_i}: term c x^a becomes c y^a t^e, e = <a, v_k> + lift(a) - beta_i
 * (0 on the cell's terms, > 0 on the others), every e divided by the cell's
 * smallest positive one (a change of the parameter: the same paths, and a
 * t-derivative bounded at t = 0).  At t = 0 the cell's binomial system
 * c_{a_i} y^{a_i} + c_{b_i} y^{b_i} = 0 remains, with |det D| solutions; at
 * t = 1 every cell's homotopy is g, and the paths of all cells end at the
 * isolated roots of g in (C*)^n.  phc_num_paths reports the sum of the
 * volumes; paths are numbered cell by cell in the given order.  Only
 * phc_polyhedral_starts, phc_track_polyhedral, phc_refine_endpoints and
 * phc_num_paths accept the handle.
 * Errors: as phc_make_homotopy; PHC_EINVAL for n_cells < 1, a NULL cell
 * list, a cell that is not a fine mixed cell of this lifting, or a zero
 * coefficient on a cell's term; PHC_EUNSUPPORTED when a cell's exact data
 * overflow. */
int phc_make_polyhedral_homotopy(int n, const int32_t *terms_per_eq, const uint8_t *exps, const phc_cd *coefs,
                                 const int32_t *lift, const int32_t *cells, int64_t n_cells, phc_homotopy **out);

/* Start solutions of paths first_path .. first_path+n_paths-1 of a
 * polyhedral handle to x_out (device SoA [n][n_paths]): the solutions of
 * the cell's binomial system y^D = beta, beta_i = -c_{a_i} / c_{b_i}, from
 * the Hermite form U D = H (U unimodular, H upper triangular with a positive
 * diagonal): log y_k = (sum_j U_kj log beta_j - sum_{l>k} H_kl log y_l
 * + 2 pi i r_k) / H_kk for k = n-1 .. 0, with r_k the digits of the path's
 * index within its cell in the radices H_00 .. H_(n-1)(n-1) (r_0 fastest).
 * Errors: PHC_EINVAL for a handle of another kind, a range outside the
 * paths or a NULL x_out; PHC_ECUDA. */
int phc_polyhedral_starts(const phc_homotopy *h, int64_t first_path, int64_t n_paths, phc_cd *x_out,
                          void *cuda_stream);

/* Track paths first_path .. first_path+n_paths-1 of a polyhedral handle from
 * their start solutions at t = 0 to t = 1, with the readings of
 * phc_track_paths (RK4 predictor, Newton corrector, step control, end Newton
 * at t = 1, classification against g), one thread per path; outputs as
 * phc_track_paths (x_out SoA [n][n_paths], cls_out, stats_out or NULL).  No
 * tail hand-off and no compaction (tail_drain and compact do not apply).
 * Errors: as phc_track_paths; PHC_EINVAL for a handle of another kind. */
int phc_track_polyhedral(phc_homotopy *h, int64_t first_path, int64_t n_paths, const phc_opts *opts,
                         phc_cd *x_out, int8_t *cls_out, phc_path_stats *stats_out, void *cuda_stream);

/* Solve a system g with coefficients in general position by polyhedral
 * homotopies in the two-stage pipeline of Section 2.2 (Figure 2): the calling
 * thread makes the mixed cells one after the other (as phc_mixed_cells with
 * lift) while the GPU already tracks the paths of the cells made so far
 * (batches of cells of growing size, launched as they are made on helper
 * streams with the priority of cuda_stream); the endpoints are classified
 * against g at the end.  Outputs (device): x_out SoA [n][max_paths], cls_out
 * [max_paths], stats_out [max_paths] or NULL; paths are numbered cell by
 * cell in the order the cells were made (the order phc_mixed_cells
 * reports), so the results equal those of phc_track_polyhedral on a handle
 * over those cells.  *n_paths_out: the mixed volume; *n_cells_out (may be
 * NULL): the number of cells.  Host call: returns once the work on
 * cuda_stream has finished.
 * Errors: as phc_mixed_cells and phc_make_polyhedral_homotopy; PHC_EINVAL
 * when the mixed volume exceeds max_paths (*n_paths_out still reports it;
 * the outputs are then incomplete); PHC_ENOMEM; PHC_ECUDA. */
int phc_solve_polyhedral(int n, const int32_t *terms_per_eq, const uint8_t *exps, const phc_cd *coefs,
                         const int32_t *lift, const phc_opts *opts, int64_t max_paths, phc_cd *x_out,
                         int8_t *cls_out, phc_path_stats *stats_out, int64_t *n_paths_out, int64_t *n_cells_out,
                         void *cuda_stream);

/* Message of the last non-OK return on the calling thread ("" if none). */
const char *phc_last_error(void);

void phc_destroy_homotopy(phc_homotopy *h);
void phc_free_lists(phc_system_lists *lists);

/* Sizes of the structs, for bindings that mirror them. */
int phc_sizeof_opts(void);
int phc_sizeof_stats(void);

#ifdef __cplusplus
}
#endif

#endif /* PHC_H */
