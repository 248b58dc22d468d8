/*
 * fiesta.h -- C ABI of the GB300 sector-integrand Monte-Carlo library.
 *
 * The library integrates sector-decomposed, eps-expanded Feynman-parameter
 * integrands (the "units": one sector at one power of eps) with the VEGAS
 * algorithm on one GPU.  It is the device half of the method of A. V. Smirnov,
 * "FIESTA 4: optimized Feynman integral calculations with GPU support"
 * (arXiv:1511.03614): Sec. 2.1-2.2 describe evaluating each integrand as a
 * loop over (operator, operand, operand, result) quadruples at batches of
 * sampling points on the GPU; Sec. 4.4 names Vegas the default integrator;
 * Sec. 4.3 reports per eps order a value and an error estimate, the errors of
 * the separately integrated pieces summed in the mean-square norm.
 *
 * Conventions for every entry point:
 *  - Plain C types only.  All arrays are owned by the caller unless stated.
 *  - A return value of 0 (FIESTA_OK) means success; a negative value is one of
 *    the FIESTA_E_* codes below and fiesta_last_error() returns a message
 *    (thread-local, valid until the next call on the same thread).
 *  - Nothing of the integration is computed on the host: if no usable GPU is
 *    present every entry point that would evaluate integrands returns
 *    FIESTA_E_CUDA.  The accuracy loop's bookkeeping (fiesta_assemble,
 *    fiesta_allocate_points) is plain host arithmetic on a few numbers per result.
 */
#ifndef FIESTA_H
#define FIESTA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FIESTA_OK            0
#define FIESTA_E_INVALID    -1  /* bad argument or program rejected by the validator */
#define FIESTA_E_NOMEM      -2  /* device memory or shared memory budget exceeded */
#define FIESTA_E_CUDA       -3  /* CUDA runtime error (message has the CUDA text) */
#define FIESTA_E_TIMEOUT    -4  /* device time budget expired; the kernel stopped cleanly */
#define FIESTA_E_NONFINITE  -5  /* a unit produced non-finite samples (unit id in the message) */

#define FIESTA_RNG_PHILOX    0
#define FIESTA_RNG_SOBOL     1
#define FIESTA_FP64          0  /* all arithmetic in binary64 */
#define FIESTA_FP32          1  /* integrand body and map in binary32; sums, Vegas histogram and grid in
                                   binary64; points with a coordinate below small_x32 in binary64 */
#define FIESTA_AUTO          2  /* per unit: binary32 where a probe against binary64 stays within budget */
#define FIESTA_DD            3  /* fiesta_eval_batch only: every point in double-double (about 106 bits) */

#define FIESTA_PROPOSAL_VEGAS 0  /* sampling points from the Vegas map of each unit */
#define FIESTA_PROPOSAL_FLOW  1  /* sampling points from each unit's normalising flow (learned proposal) */

#define FIESTA_METHOD_VEGAS  0  /* fiesta_integrate_to_accuracy: Vegas iterations (either proposal) */
#define FIESTA_METHOD_RQMC   1  /* adapted Vegas grids, then digitally shifted Sobol replicates */
#define FIESTA_METHOD_CUHRE  2  /* adaptive cubature with a shrinking per-unit tolerance */

#define FIESTA_NBINS       128  /* Vegas bins per coordinate */
#define FIESTA_MAX_DIM       8  /* largest integration dimension */
#define FIESTA_MAX_OUT       6  /* results (eps orders) of one fused unit */

/*
 * One unit: a straight-line register program (the paper's quadruple list,
 * Sec. 2.1) plus its constants.  Instruction word: op | dst<<8 | a<<16 | b<<24,
 * opcodes 1..16 as documented in the Python package's bytecode module
 * (LDX LDC ADD SUB MUL DIV NEG MAC ADDC MULC MACC POWI LOG INV MOV ATAN2).
 * code/consts are host pointers, read during fiesta_load_sectors only.
 */
typedef struct {
    int32_t dim;          /* integration dimension, 1..FIESTA_MAX_DIM */
    int32_t n_instr;      /* number of instruction words, >= 1 */
    int32_t n_const;      /* number of constants, 0..49152 */
    int32_t n_slots;      /* register-file size, 1..255 */
    int32_t out_slot;     /* slot holding the integrand value at the end */
    int32_t order;        /* power of eps of this unit (used for the per-order sums) */
    int32_t sector;       /* sector number (informational) */
    uint32_t rng_key;     /* second Philox key word: the unit's point stream */
    const uint32_t *code; /* n_instr words */
    const double *consts; /* n_const values */
    int32_t n_out;        /* 0 or 1: one result in out_slot; 2..FIESTA_MAX_OUT: a fused unit whose
                             results are the eps orders order .. order + n_out - 1 (vector-valued
                             integrand sharing one Vegas grid), in out_slots */
    const int32_t *out_slots; /* n_out slots (when n_out > 1) */
    int32_t cplx;         /* nonzero: a contour-deformed unit whose results are (re, im) pairs,
                             result 2k + p being part p of eps order order + k */
} fiesta_program;

/* Optional device allocator (e.g. a framework's caching allocator).  NULL
 * members select cudaMalloc/cudaFree. */
typedef struct {
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, void *user);
    void *user;
} fiesta_alloc;

typedef struct {
    int32_t rng;              /* FIESTA_RNG_PHILOX or FIESTA_RNG_SOBOL */
    int32_t precision;        /* FIESTA_FP64 or FIESTA_FP32 */
    int32_t n_iter;           /* Vegas iterations, >= 1 */
    int32_t adapt;            /* 1: refine each unit's grid between iterations; 2: also after the last one */
    int64_t points_per_iter;  /* sampling points per unit per iteration, >= 2 */
    uint64_t seed;            /* first Philox key word is seed mod 2^32 */
    double alpha;             /* grid damping exponent (1.5) */
    int32_t skip_first;       /* nonzero: leave iteration 0 out of the weighted mean */
    int32_t order_lo;         /* value[k], error[k] refer to eps^(order_lo + k) */
    int64_t unit_begin;       /* integrate units [unit_begin, unit_end) only ... */
    int64_t unit_end;         /* ... unit_end <= 0 means all units */
    int64_t timeout_ms;       /* device time budget per kernel launch; 0 = none */
    int32_t threads;          /* threads per block (multiple of 32, <= 512; <= 384 when fused units keep
                                 their sums in shared memory; a power of two with Sobol); 0 = autotuned,
                                 which also splits a precision's units by slot count (see
                                 fiesta_stats.wide_threads) */
    int32_t reset_grid;       /* nonzero: start from the uniform grid (else keep the last one) */
    int32_t iter_offset;      /* added to the iteration number in the point streams */
    int32_t points_per_thread;/* points per thread per work item; 0 = autotuned */
    int64_t probe_points;     /* FIESTA_AUTO: probe points per unit (0: 16384) */
    double fp32_budget;       /* FIESTA_AUTO: largest relative error of a unit's mean accepted in binary32 (0: 1e-6) */
    int32_t no_graph;         /* nonzero: launch directly instead of replaying the iteration loop as a
                                 CUDA graph (captured on the first call, reused while the call's
                                 parameters are unchanged) */
    int32_t accumulate;       /* units with several results: where the per-thread sums of the evaluation
                                 kernel live; 0 = autotuned, 1 = registers, 2 = shared memory (both
                                 variants give the same sums up to rounding order) */
    double small_x;           /* extended precision near the boundary (the paper's mixed mode, Sec. 4.6,
                                 SmallX), where the subtraction terms cancel: > 0 evaluates every
                                 point of a binary64 unit with a coordinate below small_x in
                                 double-double; 0 = off.  Units with complex results are rejected
                                 when it is set. */
    const int64_t *unit_points;  /* nullable host array, one entry per unit of the slice: points per
                                 iteration of that unit (>= 2; <= 2^32 with Sobol), replacing
                                 points_per_iter (which still sizes the autotuner's trials).  Lets a
                                 caller spend points where the variance is (see the binding's
                                 run_to_accuracy); the point streams do not depend on it. */
    double small_x32;         /* the same one level down: > 0 evaluates every point of a binary32
                                 unit with a coordinate below small_x32 in binary64 (the
                                 subtraction differences near the boundary stay binary64), and the
                                 FIESTA_AUTO probe counts such points as exact for binary32; 0 = off.
                                 The Python binding passes 2^-20 for binary32 and AUTO: below it a
                                 coordinate's terms fall under half a binary32 ulp of the corner
                                 polynomials, so f(t) - f(t|t_j=0) would vanish instead of giving
                                 its finite limit (a bias, not noise). */
    int32_t proposal;         /* FIESTA_PROPOSAL_VEGAS (0) or FIESTA_PROPOSAL_FLOW: each iteration then
                                 draws its points from the units' flows (fiesta_flow_*; initialised
                                 with seed on first use), precision FIESTA_FP64 or FIESTA_FP32, Philox
                                 points; between iterations the flows are trained flow_train_steps
                                 Adam steps on flow_keep points per unit kept from the iteration;
                                 iterations are combined as Vegas iterations are.  adapt, rng,
                                 unit_points and small_x do not apply. */
    int32_t flow_train_steps; /* FLOW: training steps after every iteration but the last (0: none) */
    int64_t flow_keep;        /* FLOW: points kept per unit for training (0: 4096) */
    double flow_lr;           /* FLOW: Adam learning rate (0: 2e-3) */
    int32_t flow_power;       /* FLOW: loss weights (|f|/q)^power (0: 1, the KL divergence) */
    int32_t wide_threads;     /* > 0: split each precision's units by slot count whenever the
                                 largest slot file does not fit a 512-thread block (as the autotuner
                                 does) and run the units whose files fit with this many threads per
                                 block (multiple of 32, <= 512); points_per_thread, when given, applies
                                 to both groups.  0: split only when the shape is autotuned. */
} fiesta_options;

typedef struct {
    double value;             /* inverse-variance weighted mean over iterations */
    double sigma;             /* its standard error */
    double chi2_dof;          /* chi^2 per degree of freedom of the iterations */
    int64_t n_points;         /* points evaluated for this unit */
    int32_t order, sector;
    int64_t n_nonfinite;      /* samples whose value was not finite (counted as 0) */
    int32_t precision;        /* FIESTA_FP64 or FIESTA_FP32: how this unit was evaluated */
    int32_t unit;             /* unit index (a fused unit gives one record per result) */
    int32_t part;             /* complex units: 0 real part, 1 imaginary part */
    int32_t pad;
    double fp32_error;        /* FIESTA_AUTO: probe estimate of the binary32 error of the mean (else NaN) */
} fiesta_unit_result;

typedef struct {
    double gpu_ms;            /* device time of all launches (CUDA events) */
    double eval_ms;           /* device time of the evaluation kernel alone */
    int64_t points;           /* sampling points evaluated */
    double points_per_s;      /* points / (gpu_ms / 1000) */
    int32_t kernels_launched; /* kernel launches made by this call */
    int32_t eval_launches;    /* of which evaluation-kernel launches */
    int64_t units_fp32;       /* units evaluated in binary32 */
    int64_t unit_points;      /* evaluations of (sector, order) integrands: points x results, a
                                 complex unit's (re, im) pair counting as one */
    int32_t threads[2];       /* block size used for binary64 [0] and binary32 [1] (when a precision's
                                 units were split by slot count: that of the units with the most slots) */
    int32_t points_per_thread[2];
    int64_t points_ext;       /* points promoted near the boundary (small_x: binary64 -> double-double,
                                 small_x32: binary32 -> binary64) */
    int32_t wide_threads[2];  /* block size of the units with few slots when a precision's units
                                 were split by slot count (their slot files fit 512-thread blocks and the
                                 others' do not); 0: not split */
    int32_t wide_points_per_thread[2];
    int32_t eval_groups;      /* evaluation launches per iteration (one per precision and slot group) */
    int32_t pad;
} fiesta_stats;

typedef struct fiesta_ctx fiesta_ctx;

/*
 * Copy n_units programs to the device and validate them (opcodes, slot,
 * coordinate and constant indices, read-before-write).  *out receives a new
 * context, owned by the caller and released by fiesta_free.  cuda_stream is a
 * cudaStream_t (NULL: the default stream) on which every later call runs.
 * Errors: FIESTA_E_INVALID (a program is rejected, index in the message),
 * FIESTA_E_NOMEM, FIESTA_E_CUDA.
 */
int fiesta_load_sectors(fiesta_ctx **out, const fiesta_program *progs, int64_t n_units,
                        const fiesta_alloc *alloc, void *cuda_stream);

/*
 * Integrate every unit of the slice with Vegas (Sec. 4.4) and return, per eps
 * order order_lo + k (k < n_orders), the sum over units of that order (real
 * parts; imaginary parts of complex units are in the per-unit records) in
 * value[k] and the mean-square combination sqrt(sum sigma^2) of their errors
 * in error[k] (Sec. 4.3).  value/error are caller-owned host arrays of
 * n_orders doubles.  per_unit (nullable) receives one record per result of the
 * slice's units (one per unit, n_out per fused unit), in unit order; stats
 * (nullable) the timing.  The grids persist in the
 * context between calls (see reset_grid).
 * Errors: FIESTA_E_INVALID, FIESTA_E_CUDA, FIESTA_E_TIMEOUT, FIESTA_E_NONFINITE
 * (results are still written; the message names the first unit affected).
 */
int fiesta_integrate(fiesta_ctx *ctx, const fiesta_options *opt, double *value, double *error,
                     int32_t n_orders, fiesta_unit_result *per_unit, fiesta_stats *stats);

/*
 * Integrate until every eps order n of the assembled series R_n = sum_m c_m I_(n-m)
 * (I_K the per-order sums over units, c the caller's prefactor series) has an error
 * at most target * max(|R_n|, floor * max_k |R_k|) -- the accuracy loop of the
 * paper's pool (Sec. 4.5-4.6: integrate, check the error, continue), on the device
 * side.  Methods:
 *  FIESTA_METHOD_VEGAS: calls of fiesta_integrate with iters_per_call iterations
 *    (grids kept and refined between calls, iteration numbers continuing); every
 *    iteration but the first `skip` enters a per-result inverse-variance combination;
 *    with allocate, the points of each later call go to the units by Neyman
 *    allocation for the assembled series (unit u's per-point spread s_uK, cost per
 *    point w_u = program length + 4 dim + 8, N_u proportional to
 *    sqrt(max_n (sum_K |c_(n-K)| s_uK / tau_n)^2 / w_u), total cost unchanged, each
 *    N_u within [0.01, 64] x points).  With proposal FLOW each round draws `points`
 *    from the flows (keeping `keep` per unit for training during the first
 *    train_rounds rounds, then steps_per_round Adam steps); rounds from `skip` on are
 *    combined.
 *  FIESTA_METHOD_RQMC: adapt_iters Philox iterations adapt the grids (adapt_points
 *    points, 0: points); then each round integrates every unit with `replicates`
 *    independent digital shifts of a Sobol sequence of N points (N = points, doubled
 *    every round up to max_points) on the frozen grids; a result's round estimate is
 *    the replicate mean, its variance the replicates' sample variance / replicates;
 *    rounds are combined with inverse-variance weights.
 *  FIESTA_METHOD_CUHRE: fiesta_cuhre with per-unit tolerance rel_tol (0: target),
 *    multiplied by shrink (0: 0.1) after every attempt that misses the target; errors
 *    are bounds and add linearly.
 * A call continues from `state` (caller-owned, zeroed for a fresh start): sw, swi
 * (one entry per result of every unit, n_out per unit in unit order) and n_used (one
 * per unit) are read and updated, so a caller can stop (max_calls), save the state
 * and resume with the same point streams.  Outputs (host arrays, caller-owned):
 * value/error per assembled order out_lo + k, k < n_out_orders (real parts and their
 * errors; value_im/error_im, nullable, the imaginary parts of problems with complex
 * units), unit_value/unit_sigma (nullable) per result.  The ratio max_n error/target
 * and the converged flag are in state.  Errors: those of the calls it makes.
 */
typedef struct {
    int32_t method;            /* FIESTA_METHOD_* */
    int32_t proposal;          /* METHOD_VEGAS: FIESTA_PROPOSAL_VEGAS or FIESTA_PROPOSAL_FLOW */
    int32_t precision;         /* FIESTA_FP64, FIESTA_FP32 or FIESTA_AUTO (flow: FP64 or FP32) */
    int32_t allocate;          /* METHOD_VEGAS, Vegas proposal: Neyman allocation across units */
    double target;             /* relative error per order of the assembled series, > 0 */
    double floor;              /* order n is judged against max(|R_n|, floor * max_k |R_k|) */
    int64_t points;            /* points per unit per iteration (RQMC: the first Sobol length) */
    int32_t iters_per_call;    /* METHOD_VEGAS: iterations per fiesta_integrate call (0: 2) */
    int32_t max_iters;         /* iteration (flow, RQMC: round; cubature: attempt) cap */
    int32_t skip;              /* leading iterations (flow rounds) left out of the combination */
    int32_t max_calls;         /* METHOD_VEGAS: return after this many calls (0: no limit) */
    uint64_t seed;
    double max_gpu_s;          /* return once this much device time is spent (0: no cap) */
    double small_x, small_x32; /* as in fiesta_options */
    const double *pre;         /* prefactor series c_i (host, n_pre values): c(eps) = sum c_i eps^(i - pre_q) */
    int32_t n_pre;
    int32_t pre_q;
    int32_t correlated;        /* nonzero: the assembled errors add linearly (fused units' orders are correlated) */
    int32_t out_lo;            /* value[k] refers to eps^(out_lo + k) */
    int32_t replicates;        /* RQMC: digital shifts per round (0: 8) */
    int32_t adapt_iters;       /* RQMC: Philox iterations adapting the grids (0: 6) */
    int64_t adapt_points;      /* RQMC: points per unit of those iterations (0: points) */
    int64_t max_points;        /* RQMC: largest Sobol length per replicate (0: 2^22) */
    int32_t train_rounds;      /* FLOW: rounds with training (0: 8) */
    int32_t steps_per_round;   /* FLOW: Adam steps per training round (0: 20) */
    double lr;                 /* FLOW: learning rate (0: 2e-3) */
    int32_t power;             /* FLOW: loss weight exponent (0: 1) */
    int32_t reserved;
    int64_t keep;              /* FLOW: points kept per unit for training (0: 4096) */
    double rel_tol;            /* CUHRE: first per-unit tolerance (0: target) */
    double shrink;             /* CUHRE: tolerance factor per missed attempt (0: 0.1) */
    int32_t max_passes;        /* CUHRE: passes per attempt (0: 60) */
    int32_t reserved2;
    int64_t max_regions;       /* CUHRE: region limit per attempt (0: 2^22) */
} fiesta_accuracy_options;

typedef struct {
    double *sw, *swi;          /* per result: running sums of 1/var and mean/var (caller-owned) */
    double *n_used;            /* per unit: points counted so far (caller-owned) */
    int32_t iterations;        /* iterations, rounds or attempts done */
    int32_t converged;         /* every order met its target */
    double gpu_ms;             /* device time of all calls so far */
    int64_t points;            /* (sector, order) integrand evaluations so far */
    double ratio;              /* max over orders of |error| / target after the last check */
    int64_t points_per_replicate; /* RQMC: the last Sobol length */
    double rel_tol;            /* CUHRE: the last per-unit tolerance */
    double *order_sw, *order_swi; /* RQMC, nullable (caller-owned, 2 * n_out_orders entries each: the
                                 real parts, then the imaginary parts): per assembled order,
                                 running sums of 1/var and mean/var of the assembled series
                                 formed replicate by replicate.  When set, rounds are combined
                                 per assembled order, so the correlation of a fused unit's orders
                                 (evaluated at the same points) enters the error as measured
                                 instead of through opt->correlated's bound; the per-result
                                 sums sw, swi are kept as well. */
} fiesta_accuracy_state;

int fiesta_integrate_to_accuracy(fiesta_ctx *ctx, const fiesta_accuracy_options *opt, fiesta_accuracy_state *state,
                                 int32_t n_out_orders, double *value, double *error, double *value_im,
                                 double *error_im, double *unit_value, double *unit_sigma);

/*
 * The two arithmetic steps of that loop as plain host functions (no GPU, no
 * context), used by it and exposed so that they can be checked on their own.
 * fiesta_assemble: per-order sums of n_rec results (eps order order[k], part[k] 0
 *   real / 1 imaginary, value val[k], error sig[k]) -- errors in the mean-square norm
 *   (Sec. 4.3), or added when `linear` (error bounds) -- then the prefactor series of
 *   opt (pre, n_pre, pre_q, correlated, out_lo): value/error (and value_im/error_im,
 *   nullable) for the assembled orders out_lo .. out_lo + n_out - 1; *ratio
 *   (nullable) = max_n |error_n| / (target * max(|R_n|, floor * max_k |R_k|)).
 * fiesta_allocate_points: the Neyman allocation of the loop above for n_units units
 *   of cost cost[u] per point (program length + 4 dim + 8 in the loop), from the
 *   results' errors sig[k] (rec_unit[k], rec_order[k]), the points each unit has used
 *   (n_used) and the assembled values (value, value_im nullable: n_out orders from
 *   out_lo) that set the targets; points[u] receives the allocation.
 * Errors: FIESTA_E_INVALID.
 */
int fiesta_assemble(const fiesta_accuracy_options *opt, int64_t n_rec, const int32_t *order, const int32_t *part,
                    const double *val, const double *sig, int32_t linear, int32_t n_out, double *value,
                    double *error, double *value_im, double *error_im, double *ratio);
int fiesta_allocate_points(const fiesta_accuracy_options *opt, int64_t n_units, const double *cost, int64_t n_rec,
                           const int64_t *rec_unit, const int32_t *rec_order, const double *sig,
                           const double *n_used, int32_t n_out, const double *value, const double *value_im,
                           int64_t *points);

/*
 * Evaluate unit `unit` at n points: x is n*dim coordinates in (0,1), row-major,
 * f receives n*n_out values (row-major: the unit's results per point).  x and f are both host or both device pointers (the
 * library detects which).  precision is FIESTA_FP64, FIESTA_FP32 or FIESTA_DD
 * (double-double arithmetic, results rounded to binary64; not for complex
 * units).  This is the per-point hook, the counterpart of the paper's
 * justEvaluate integrator (Sec. 4.4).  Errors: FIESTA_E_INVALID, FIESTA_E_CUDA.
 */
int fiesta_eval_batch(fiesta_ctx *ctx, int64_t unit, int32_t precision, const double *x, int64_t n,
                      double *f);

/*
 * Per-iteration results of the last fiesta_integrate call for result `out` of
 * one unit: mean[i] and var[i] (variance of the mean) for i < n_iter, host arrays.
 */
int fiesta_iterations(fiesta_ctx *ctx, int64_t unit, int32_t out, int32_t n_iter, double *mean, double *var);

/*
 * Per-unit binary32 probe (the precision policy of FIESTA_AUTO): evaluate
 * units [unit_begin, unit_end) at n_points Philox points through their
 * current grids in binary64 and in binary32 and return, per unit, the
 * relative error of the binary32 sample mean (err_mean) and the largest
 * pointwise difference divided by the mean |f J| (err_max).  Host arrays of
 * unit_end - unit_begin doubles.  The paper's counterpart is the mixed
 * MPFR/double mode of its integration workers (Sec. 4.6, MPFR/Native/Mixed).
 */
int fiesta_precision_probe(fiesta_ctx *ctx, int64_t unit_begin, int64_t unit_end, int64_t n_points, uint64_t seed,
                           double *err_mean, double *err_max);

/* Copy one unit's Vegas grid (dim * (FIESTA_NBINS+1) edges, row per coordinate)
 * to the host array `grid`, or set it from `grid` (checkpoint and resume). */
int fiesta_get_grid(fiesta_ctx *ctx, int64_t unit, double *grid);
int fiesta_set_grid(fiesta_ctx *ctx, int64_t unit, const double *grid);

/* Apply one Vegas refinement (smoothing, damping, re-binning) to `n` grids
 * of dimension `dim` from their v^2 histograms, on the device: grid is
 * n*dim*(NB+1) edges, hist n*dim*NB sums, both host arrays; grid is updated
 * in place.  Exposed so the refinement step can be checked on its own. */
int fiesta_refine(fiesta_ctx *ctx, int32_t dim, int64_t n, double alpha, double *grid, const double *hist);

/*
 * Deterministic adaptive cubature, the Cuhre alternative to Vegas among the
 * integrators of Sec. 4.4 (CurrentIntegrator = cuhreCuba).  The paper does not
 * describe it; the library uses the degree-7 rule of Genz and Malik (J. Comput.
 * Appl. Math. 6 (1980) 295) with its embedded degree-5 rule, region error
 * |I7 - I5| per result, and splits a region in halves across the coordinate
 * with the largest fourth difference (summed over the unit's results; ties go
 * to the wider side, then the lower coordinate).  Subdivision runs in passes
 * over all live regions of all units of the slice at once: evaluate every live
 * region; a unit whose summed error is <= tau for every result stops; in the
 * other units a region whose error is <= tau * its volume (for every result) is
 * frozen and the others are split.  tau_o = max(abs_tol, rel_tol * |estimate_o|),
 * the modulus of the (re, im) pair for complex units.  Units of dimension 1 are
 * integrated as 2-dimensional ones that ignore the second coordinate.
 *
 * rel_tol, abs_tol: tolerances (> 0 and >= 0).  max_passes: pass limit (0: 40).
 * max_regions: limit on frozen + live regions of the call (0: 2^22); when the
 * next pass would exceed it, the call stops with the current estimates.
 * order_lo, unit_begin, unit_end: as in fiesta_options.  timeout_ms: checked
 * between passes (0: none).  threads: block size of the evaluation kernel
 * (0: 128; a multiple of 32, <= 256).
 */
typedef struct {
    double rel_tol;
    double abs_tol;
    int32_t max_passes;
    int32_t order_lo;
    int64_t max_regions;
    int64_t unit_begin;
    int64_t unit_end;
    int64_t timeout_ms;
    int32_t threads;
    int32_t reserved[3];
} fiesta_cuhre_options;

/* One record per result of a unit (n_out per unit, in unit order). */
typedef struct {
    double value;             /* estimate: sum over frozen and live regions of I7 */
    double error;             /* sum of the regions' |I7 - I5| */
    int64_t n_regions;        /* frozen + live regions of the unit at the end */
    int64_t n_points;         /* integrand evaluations spent on the unit */
    int32_t order;            /* eps order of the result */
    int32_t sector;
    int32_t unit;
    int32_t part;             /* complex units: 0 real, 1 imaginary part */
    int32_t converged;        /* the unit met its tolerances */
    int32_t passes;           /* passes in which the unit had live regions */
} fiesta_cuhre_result;

/*
 * Run the cubature on units [unit_begin, unit_end).  value/error (caller-owned
 * host arrays of n_orders doubles) receive per eps order order_lo + k the sum
 * over units of the estimates (real parts) and the sum of their error
 * estimates (the regions' errors are bounds, so they add linearly).  per_result
 * (nullable, host) receives one record per result of the slice's units; stats
 * (nullable) the device time and evaluations.  Device buffers are allocated
 * through the context's allocator and kept for later calls.
 * Errors: FIESTA_E_INVALID (bad options or slice), FIESTA_E_NOMEM,
 * FIESTA_E_CUDA, FIESTA_E_TIMEOUT and FIESTA_E_NONFINITE (results are still
 * written).
 */
int fiesta_cuhre(fiesta_ctx *ctx, const fiesta_cuhre_options *opt, double *value, double *error,
                 int32_t n_orders, fiesta_cuhre_result *per_result, fiesta_stats *stats);

/*
 * The regions of unit `unit` evaluated in the last pass of the last
 * fiesta_cuhre call and not split since (a unit that converged in an earlier
 * pass has none).  Up to `cap` regions are written to the host arrays center and
 * half (cap * m doubles each, m = max(dim, 2): the region is the box
 * prod [center_j - half_j, center_j + half_j]), value and error (cap * n_out:
 * I7 and |I7 - I5| per result) and axis (cap: the coordinate it would be split
 * across); *n receives the number of such regions.  Exposed so that each
 * region's rule can be checked on its own.  Errors: FIESTA_E_INVALID.
 */
int fiesta_cuhre_regions(fiesta_ctx *ctx, int64_t unit, int64_t cap, double *center, double *half, double *value,
                         double *error, int32_t *axis, int64_t *n);

/*
 * Measurement support (no counterpart in the paper): measured throughput of
 * the arithmetic pipes on the current device, used to turn an integrand's
 * instruction mix into a lower bound on its evaluation time.  out (host, >= 7
 * doubles): [0] binary64 FMA TFLOP/s, [1] binary64 log (CUDA's) G/s, [2]
 * binary64 divide G/s, [3] binary32 FMA TFLOP/s, [4] binary32 logf G/s, [5]
 * binary32 divide G/s, [6] the interpreter's table-driven binary64 log G/s,
 * when n >= 8, [7] binary64 atan2 G/s, and when n >= 9, [8] the interpreter's
 * binary64 reciprocal (Newton-Raphson refinement) G/s.
 * Allocates and frees small scratch buffers.
 */
int fiesta_probe_peaks(double *out, int32_t n);

/*
 * One Vegas sampling pass that allocates no device memory (the paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc or an allocator while they run, for example code that must not
 * synchronise the device, runs with a memory pool fixed at start-up, or has no
 * allocator hooked up).  It evaluates units [unit_begin, unit_end) of ctx at
 * `points` points each on their current grids (no adaptation) with the point
 * stream of (seed, unit, iteration), like iteration `iteration` of
 * fiesta_integrate with adapt = 0, and writes each unit's sample mean of
 * v = f*J to mean[k] and its variance of the mean to var[k], k = unit -
 * unit_begin.  mean and var are caller-owned, both host or both device arrays.
 * The context's device must be the current device.
 *
 * Non-finite samples count as zero, as in fiesta_integrate.  With host arrays
 * the call waits for the GPU and then returns FIESTA_E_NONFINITE (the first such
 * unit named in the message; mean and var are still written).  With device
 * arrays the call does not wait, so it cannot return that status: instead the
 * variance of every unit whose samples were not all finite is set to NaN.  Host
 * arrays need that wait, which stream capture forbids: during a capture only
 * device arrays are accepted.
 *
 * Its scratch (partial sums, counters) is one file-scope device array of
 * 1 966 112 bytes (about 1.97 MB) that every GPU loading the library keeps until
 * the process exits.  Limits: at most 16384 units and 65536 work items (items
 * of 2048 points) per call; larger requests return FIESTA_E_INVALID with the
 * sizes in the message.  The first call on each device looks up the array's
 * device address (a CUDA runtime query, no allocation); make that first call
 * before any stream capture.  All calls share the array and it keeps the last
 * call's contents; the parts that must start at zero are cleared by each call.
 * Calls whose work overlaps on the GPU (other streams, other threads) race on
 * the array.
 * Errors: FIESTA_E_INVALID, FIESTA_E_CUDA, FIESTA_E_NOMEM (shared memory),
 * FIESTA_E_NONFINITE (host arrays only).
 */
int fiesta_sample_noalloc(fiesta_ctx *ctx, int64_t unit_begin, int64_t unit_end, int64_t points, uint64_t seed,
                          int32_t iteration, int32_t precision, int32_t rng, double *mean, double *var);

/*
 * Learned proposal (not in the paper): per unit, a normalising flow over the
 * unit cube that stands in for the Vegas map.  Four affine coupling layers in
 * logit space, each with an MLP 16 -> 64 -> 64 -> 16 (ReLU); the sampler runs
 * the MLPs on the tensor cores in BF16 with FP32 accumulation; training
 * computes the gradient on the tensor cores too (forward and reverse-mode
 * products of the MLPs as BF16 MMAs with FP32 accumulation) and updates
 * binary32 master weights with Adam.  Parameters: FIESTA_FLOW_PARAMS floats per unit, per
 * layer W1[16][64], b1[64], W2[64][64], b2[64], W3[64][16] (outputs 0..7 the
 * scales, 8..15 the shifts), b3[16].
 *
 * fiesta_flow_init: allocate the flows of every unit of ctx (about 450 KB per
 *   unit with the Adam state and the packed copy) and initialise them to the
 *   identity map (zero output layer, random hidden layers, Philox seeded).
 * fiesta_flow_params: copy one unit's binary32 parameters to (set = 0) or from
 *   (set != 0) the host array `params`.
 * fiesta_flow_sample: one importance-sampling pass over units [unit_begin,
 *   unit_end): `points` points per unit from the flow (Philox stream of (seed,
 *   unit, iteration)), the integrand evaluated in `precision`; writes the mean
 *   of f/q and its variance of the mean to host arrays mean, var, one entry per
 *   result of the slice's units (n_out per unit, in unit order).  The first
 *   `keep` points of each unit are kept for training, with |f| (the norm of the
 *   result vector for units with several results) as the training target.
 * fiesta_flow_train: `steps` Adam steps (learning rate lr) on the kept points,
 *   loss -sum_i w_i log q(x_i) with w_i proportional to (|f_i|/q_i)^power (one
 *   flow per unit: a fused unit's orders share it)
 *   (power 1: KL divergence, 2: variance); `loss` (nullable, host) receives the
 *   last step's loss per unit.
 * fiesta_flow_check: parity hook for one unit: the sampler at the caller's base
 *   points z (n x dim, host) gives x, log q and f; the training pass at those x
 *   with the caller's weights w gives log q, the loss and its gradient
 *   (FIESTA_FLOW_PARAMS floats), computed as fiesta_flow_train computes them.
 *   All arrays host.
 * Errors: FIESTA_E_INVALID, FIESTA_E_NOMEM, FIESTA_E_CUDA, FIESTA_E_NONFINITE.
 */
#define FIESTA_FLOW_PARAMS 25152
int fiesta_flow_init(fiesta_ctx *ctx, uint64_t seed, double init_scale);
int fiesta_flow_params(fiesta_ctx *ctx, int64_t unit, float *params, int32_t set);
int fiesta_flow_sample(fiesta_ctx *ctx, int64_t unit_begin, int64_t unit_end, int64_t points, uint64_t seed,
                       int32_t iteration, int32_t precision, int64_t keep, double *mean, double *var,
                       fiesta_stats *stats);
int fiesta_flow_train(fiesta_ctx *ctx, int64_t unit_begin, int64_t unit_end, int32_t steps, double lr, int32_t power,
                      double *loss, fiesta_stats *stats);
int fiesta_flow_check(fiesta_ctx *ctx, int64_t unit, int64_t n, int32_t precision, const double *z, double *x,
                      double *logq, double *f, const double *w, double *logq_train, double *loss, float *grad);

void fiesta_free(fiesta_ctx *ctx);
const char *fiesta_last_error(void);
int fiesta_version(void);

/* The forwarded program the evaluation kernels execute for one program, for checking
 * on the host (no counterpart in the method; host only, no device call).  The program is
 * validated as fiesta_load_sectors does.  Each 64-bit word is one executed instruction:
 * bits 0-7 the opcode, 8-15 the destination slot, 16-31, 32-47 and 48-63 the operand
 * references X, Y, Z.  For ADD, SUB, MUL, NEG, MAC, ADDC, MULC, MACC and MOV the
 * instruction computes fma(X, Y, Z).  For DIV, POWI, LOG, INV and ATAN2, X and Y are the
 * first and second operand; for POWI, Y is the exponent byte.  A reference below 0xC000
 * is a constant index; 0xC000 + s is slot s; 0xD000 + j is coordinate j; 0xE000 + k is
 * the fixed constant -0, 1 or -1 (k = 0, 1, 2).  LDX and LDC execute nothing: their
 * readers name the coordinate or constant.  A MOV into the slot the next instruction
 * writes is folded into that instruction.  out (host, caller-owned) receives the first
 * min(count, cap) words.  Returns the word count, which is at most n_instr, or
 * FIESTA_E_INVALID. */
int64_t fiesta_micro_ops(const fiesta_program *prog, uint64_t *out, int64_t cap);

/* Sizes in bytes of this header's structures as the library was compiled, for a binding
 * to check its own layouts against (no counterpart in the method; host only, no device
 * call).  sizes (host, caller-owned, n entries) receives, as far as n reaches:
 * fiesta_program, fiesta_alloc, fiesta_options, fiesta_unit_result, fiesta_stats,
 * fiesta_accuracy_options, fiesta_accuracy_state, fiesta_cuhre_options,
 * fiesta_cuhre_result.  Returns the number of structures (9); -1 for a null array
 * with n > 0. */
int fiesta_abi_sizes(int64_t *sizes, int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* FIESTA_H */
