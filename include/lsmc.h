/*
 * lsmc.h -- C ABI of the GB300 Heston / Longstaff-Schwartz / Greeks library.
 *
 * Method (Klaisoongnoen, Brown, Thomson Brown, "Low-power option Greeks",
 * HEART '22): Monte Carlo paths of the Heston model discretised by
 * Andersen's quadratic-exponential (QE) scheme from two random inputs per
 * path and step, the exponential of the log price, then Longstaff-Schwartz
 * early exercise by a least-squares curve fit per exercise date (Sec. 2.2 and
 * Sec. 2.2.1; the loop reorganisation of Sec. 4.1 is what the GPU layout
 * below replaces).  The paper names the Greeks as the purpose of the run
 * (title, Sec. 2.2) without a method; here they are central bump-and-revalue
 * differences under common random numbers.  A full-truncation Euler
 * discretisation is offered beside QE.
 *
 * Conventions for every call:
 *   - Return value: LSMC_OK (0) on success, LSMC_PENDING (1) for a request
 *     still in flight, a negative LSMC_E* code otherwise; lsmc_strerror()
 *     names it.  No C++ exception crosses this boundary.
 *   - The caller owns every struct and array it passes; the library copies
 *     what it needs before returning and keeps no caller pointer.
 *   - Pointers documented "device" are CUDA global-memory addresses on the
 *     context's device; "host" pointers are ordinary host memory.
 *   - Floating point parameters must be finite.  Model limits: S0 > 0,
 *     K > 0, T > 0, v0 >= 0, kappa > 0, theta > 0, xi >= 0 (xi > 0 for QE),
 *     |rho| <= 1, n_paths >= 1, n_steps >= 1.  Violations return
 *     LSMC_EINVAL and launch nothing.
 */
#ifndef LSMC_H
#define LSMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LSMC_ABI_VERSION 1

/* ---- status codes ------------------------------------------------------ */
#define LSMC_OK 0
#define LSMC_PENDING 1
#define LSMC_EINVAL (-1)     /* an argument is out of range or not finite */
#define LSMC_ENOMEM (-2)     /* device or workspace memory exhausted */
#define LSMC_EBUSY (-3)      /* request queue full */
#define LSMC_ETIMEOUT (-4)   /* a bounded device-side wait expired */
#define LSMC_ECUDA (-5)      /* a CUDA runtime call failed */
#define LSMC_ENOTIMPL (-6)   /* combination not supported */
#define LSMC_ENOTFOUND (-7)  /* unknown ticket */
#define LSMC_ENODEV (-8)     /* no usable CUDA device */

/* ---- enumerations ------------------------------------------------------ */
enum { LSMC_PUT = 0, LSMC_CALL = 1 };
enum { LSMC_AMERICAN = 0, LSMC_EUROPEAN = 1 };
/* Heston discretisation: Andersen QE (the paper's, Sec. 2.2) or
 * full-truncation Euler (negative variance truncated in drift and diffusion). */
enum { LSMC_SCHEME_QE = 0, LSMC_SCHEME_FT_EULER = 1 };
/* Regression basis on in-the-money paths, scaled x = S/K, w = v/theta:
 * S2 = {1, x, x^2} (the paper's quadratic curve fit, Sec. 2.2.1);
 * SV2 = {1, x, x^2, w, x w, w^2}. */
enum { LSMC_BASIS_S2 = 0, LSMC_BASIS_SV2 = 1 };
/* FP64: paths, sums, solve and estimator in double precision.
 * MIXED: paths and per-thread moment sums in single precision; cross-warp
 * sums (compensated float pairs), the normal-equation solve and the
 * estimator in double.
 * DF: paths, regression features, sums and exercise decisions in
 * unevaluated pairs of floats (about 48 significant bits, computed on the
 * FP32 pipes; the normal quantiles, the solve and the estimator in double):
 * FP64-grade results at single-precision pipe rates.  Stored values are
 * float pairs, as wide as doubles. */
enum { LSMC_FP64 = 0, LSMC_MIXED = 1, LSMC_DF = 2 };
enum { LSMC_GREEK_DELTA = 1, LSMC_GREEK_GAMMA = 2, LSMC_GREEK_VEGA = 4,
       LSMC_GREEK_RHO = 8, LSMC_GREEK_THETA = 16, LSMC_GREEK_ALL = 31 };

/* ---- value types ------------------------------------------------------- */
/* Heston model: dS = (r - q) S dt + sqrt(v) S dW1,
 * dv = kappa (theta - v) dt + xi sqrt(v) dW2, d<W1, W2> = rho dt (Sec. 2.2). */
typedef struct lsmc_heston {
  double S0, r, q, v0, kappa, theta, xi, rho;
} lsmc_heston;

typedef struct lsmc_contract {
  int32_t type;   /* LSMC_PUT / LSMC_CALL */
  int32_t style;  /* LSMC_AMERICAN (exercise dates t_1..t_N and t_0) or EUROPEAN */
  double K;       /* strike */
  double T;       /* maturity in years; exercise dates t_n = n T / n_steps */
} lsmc_contract;

/* Central bumps: S0 (1 +- rel_dS) for delta, S0 (1 +- rel_dS_gamma) for gamma
 * (0 or equal to rel_dS: gamma reuses the delta pair), v0 (1 +- rel_dv0) for
 * vega = dV/dv0, r +- abs_dr for rho, T -+ abs_dT (same n_steps) for
 * theta = -dV/dT.  greek_mask: LSMC_GREEK_* bits. */
typedef struct lsmc_bumps {
  double rel_dS, rel_dS_gamma, rel_dv0, abs_dr, abs_dT;
  uint32_t greek_mask;
  uint32_t reserved;
} lsmc_bumps;

/* Greeks not requested are NaN.  status: 0, or 1 when at least one exercise
 * date had a singular regression (no exercise there; counted in
 * n_singular_solves over all revaluations).  n_near_ties counts exercise
 * decisions (over all revaluations) whose discounted payoff lay within a
 * relative 1e-10 of the fitted continuation value: only such decisions can
 * come out differently under another rounding of the same arithmetic. */
typedef struct lsmc_result {
  double price, price_se, delta, gamma, vega, rho, theta, european_price;
  uint32_t n_singular_solves, n_revaluations;
  int32_t status;
  uint32_t n_near_ties;
} lsmc_result;

/* Bounds of one strike's American price (lsmc_price_bounds). */
typedef struct lsmc_bounds {
  double lower, lower_se;   /* out-of-sample estimator: the policy on independent paths */
  double upper, upper_se;   /* dual upper bound */
  double martingale_end;    /* mean over outer paths of the martingale at maturity */
  double martingale_end_se; /* (zero in expectation; a diagnostic) */
  double dual_ms;           /* device time of the dual pass (all strikes) */
  uint32_t n_near_ties;     /* exercise decisions within rounding reach of their threshold */
  int32_t status;           /* as lsmc_result.status */
} lsmc_bounds;

typedef struct lsmc_config {
  int32_t device;        /* CUDA device ordinal */
  int32_t precision;     /* default LSMC_FP64 / LSMC_MIXED */
  int32_t scheme;        /* default LSMC_SCHEME_QE / LSMC_SCHEME_FT_EULER */
  int32_t max_batch;     /* requests admitted together in serving; 0 = 64 */
  uint64_t hbm_budget;   /* bytes the serving loop may hold; 0 = 3/4 of free */
  uint32_t max_inflight; /* requests on the device at once (serving); 0 = 8 */
  uint32_t queue_capacity; /* pending requests accepted; 0 = 4096 */
} lsmc_config;

/* One pricing request: a family of contracts of one type/style/maturity that
 * share one path set per scenario (one per strike).  precision / scheme of
 * -1 take the context's default.  stream_id selects the random stream
 * (Philox counter word 2); seed is the Philox key. */
typedef struct lsmc_request {
  lsmc_heston model;
  int32_t type, style;
  double T;
  const double* strikes;   /* host, n_strikes values */
  uint32_t n_strikes;
  uint32_t n_paths, n_steps;
  int32_t basis;
  int32_t precision;
  int32_t scheme;
  lsmc_bumps bumps;
  uint64_t seed;
  uint32_t stream_id;
  uint32_t flags;          /* LSMC_FLAG_* (0: defaults) */
} lsmc_request;

/* lsmc_request.flags.  LSMC_FLAG_REGENERATE: keep no path store; the forward
 * pass saves the state (x, v) of every path every ceil(sqrt(n_steps)) dates,
 * and before each segment of the backward induction the segment's dates are
 * simulated again from the saved state (the random inputs are counter-based,
 * so the regenerated paths are the stored ones, bit for bit).  Device memory
 * for the paths drops from n_steps rows to about 2 sqrt(n_steps); the
 * forward work doubles.  All requests of a plan must agree on the flag and,
 * with it, on n_steps. */
enum { LSMC_FLAG_REGENERATE = 1 };
/* lsmc_request.flags.  LSMC_FLAG_OUT_OF_SAMPLE: out-of-sample
 * Longstaff-Schwartz.  The regressions run on the paths of stream_id; the
 * exercise policy they define is then applied to independent paths, the
 * same simulation on stream stream_id ^ 0x80000000, each stopping at the
 * first date where it is in the money and its discounted payoff beats the
 * fitted continuation value.  Prices, and the Greeks made from them, are the
 * means of those cash flows: low-biased estimates of the American values,
 * free of the in-sample estimator's look-ahead.  Not combined with
 * LSMC_FLAG_REGENERATE. */
enum { LSMC_FLAG_OUT_OF_SAMPLE = 2 };
/* lsmc_request.flags.  LSMC_FLAG_STORE_FP16 / LSMC_FLAG_STORE_BF16: a 16-bit
 * path store (the paper's study of reduced data types, Sec. 4.2 and Table 4,
 * applied to the stored paths only).  The forward pass computes every step in the
 * request's precision and writes exp(x) (x = log(S / S0), the path's log
 * price relative to its start) and the variance as IEEE binary16 or
 * bfloat16, rounded to nearest with ties to even; the backward induction
 * widens them exactly and works in the request's precision.  A scenario
 * reads S as its S0 times the stored value, a rate bump (which moves every
 * log price by +-dr t_n and nothing else) as the base simulation's value
 * times S0 exp(+-dr t_n).  The store takes 2 bytes per value instead of 8
 * (FP64, float pairs) or 4 (MIXED).  binary16 keeps 11 significant bits
 * (relative rounding error at most 2^-11) and overflows above 65504, i.e.
 * for x > 11.09; bfloat16 keeps 8 bits and the float range.  The two flags
 * exclude each other (LSMC_EINVAL); all requests of a plan agree on them.
 * Combines with LSMC_FLAG_REGENERATE (the segment rows are 16-bit, the saved
 * states are not) and with LSMC_FLAG_OUT_OF_SAMPLE. */
enum { LSMC_FLAG_STORE_FP16 = 4, LSMC_FLAG_STORE_BF16 = 8 };

typedef struct lsmc_ctx lsmc_ctx;
typedef struct lsmc_plan lsmc_plan;

/* ---- library ----------------------------------------------------------- */
/* Static NUL-terminated name of a status code ("unknown status" for any
 * other value).  Never fails and needs no device. */
const char* lsmc_strerror(int status);
/* LSMC_ABI_VERSION of the library actually loaded (compare it with the
 * header's to detect a mismatched build).  Never fails. */
int lsmc_abi_version(void);
/* Device allocations the library has made in this process: cudaMalloc and
 * cudaMallocAsync calls and successful lsmc_set_allocator callbacks (not the
 * sub-allocations from a workspace).  A diagnostic with no counterpart in the
 * paper: lets a caller check that a code path allocated nothing.
 * LSMC_EINVAL if count is NULL. */
int lsmc_device_allocations(uint64_t* count);

/* ---- context ----------------------------------------------------------- */
/* Creates a context on config->device (NULL: device 0, FP64, QE).  The
 * context owns a CUDA stream unless one is set, a workspace arena and, after
 * the first lsmc_submit, one scheduler thread.  Thread-safe afterwards.
 * *out (host) receives the context, owned by the caller until lsmc_destroy
 * (NULL on failure).  LSMC_EINVAL: out NULL, an unknown precision or scheme,
 * or a device ordinal out of range; LSMC_ENODEV: no CUDA device;
 * LSMC_ECUDA: the device or the context's stream could not be set up;
 * LSMC_ENOMEM: host memory. */
int lsmc_create(lsmc_ctx** out, const lsmc_config* config);
/* Waits for in-flight work, stops the scheduler, frees everything; tickets
 * not yet taken are dropped.  Destroy every plan of the context first.
 * NULL is ignored. */
void lsmc_destroy(lsmc_ctx* ctx);
/* Work of the synchronous calls runs on this CUDA stream (a cudaStream_t; NULL
 * = the context's own stream).  The caller keeps the stream alive.
 * LSMC_EINVAL if ctx is NULL. */
int lsmc_set_stream(lsmc_ctx* ctx, void* cuda_stream);
/* Device memory callbacks used instead of cudaMalloc / cudaFree for every
 * allocation the context makes outside a workspace (plans, the serving
 * arena, the dual bound's scratch): alloc(bytes, user) returns device memory
 * of the context's device, 256-byte aligned, or NULL (LSMC_ENOMEM);
 * release(ptr, user) gives it back, called only after the library's work on
 * it has completed.  This is how a framework's caching allocator (e.g.
 * PyTorch's) plugs in.  Both NULL: back to cudaMalloc.  LSMC_EBUSY once the
 * serving loop has started; LSMC_EINVAL if exactly one callback is NULL.
 * The callbacks may run on the context's scheduler thread. */
int lsmc_set_allocator(lsmc_ctx* ctx, void* (*alloc)(size_t bytes, void* user),
                       void (*release)(void* ptr, void* user), void* user);
/* Upper bound, in seconds, of every device-side wait of the context's later
 * plans and launches (a backward job waiting for the previous exercise
 * date's coefficients): on expiry the kernels record an error and return, and
 * the host call reports LSMC_ETIMEOUT; the context stays usable.  Default
 * 20 s; 0 fails any wait that is not satisfied at once.  LSMC_EINVAL outside
 * [0, 3600].  Bounded waits are a deployment safeguard (the paper has none). */
int lsmc_set_wait_limit(lsmc_ctx* ctx, double seconds);
/* Flag OR'ed into a count of sub-tiles per backward job (sub of
 * lsmc_set_backward_shape, best_sub of lsmc_autotune): in requests with
 * several strikes, the strikes in the money at the request's S0 (puts
 * struck above it, calls below) take half as many sub-tiles per job (at
 * least one) as the others.  Their regressions have the most in-the-money
 * paths per tile, so smaller jobs shorten their chain of dates, while the
 * larger jobs of the other strikes cost fewer arrivals.  Results differ only
 * by the order of the tile sums. */
#define LSMC_SUB_ITM_HALF 0x8000u
/* Tile shape of the backward pass for the context's later plans: sub
 * sub-tiles per job (optionally | LSMC_SUB_ITM_HALF) and ppt paths per
 * thread of a sub-tile (2 or 4 for LSMC_FP64 and LSMC_DF, 4 or 8 for
 * LSMC_MIXED; a value not compiled for a plan's precision falls back to its
 * default).  0, 0: chosen per plan (the autotuner's result when
 * lsmc_autotune has tuned that kind of plan).  LSMC_EINVAL for a count
 * above 64, the flag without a count, or ppt not in {0, 2, 4, 8}. */
int lsmc_set_backward_shape(lsmc_ctx* ctx, uint32_t sub, uint32_t ppt);
/* Share of the device's resident backward CTAs that one serving batch's
 * persistent backward grid takes, so that batches on different slots run
 * side by side instead of each waiting for the CTAs of the one before.
 * share in (0, 1]; 0 (the default) = 1 / config.max_inflight.  Applies to
 * batches admitted afterwards.  A serving-policy option (the paper has no
 * serving loop).  LSMC_EINVAL outside [0, 1]. */
int lsmc_set_serving_share(lsmc_ctx* ctx, double share);
/* Device memory the context sub-allocates from instead of cudaMalloc
 * (e.g. a PyTorch tensor).  Must be set before any plan exists and stay
 * valid until lsmc_destroy; 256-byte aligned.  The caller keeps ownership
 * (the library never frees it).  LSMC_EINVAL: ctx or device_ptr NULL, bytes
 * below 4096 or a misaligned pointer; LSMC_EBUSY while a plan holds part of
 * the current workspace or once the context has allocated its own arena. */
int lsmc_set_workspace(lsmc_ctx* ctx, void* device_ptr, size_t bytes);
/* Bytes of device memory a request needs (paths, regression state, tables),
 * written to *bytes (host), for the default backward shape.  Host only; ctx
 * may be NULL (then the library's default precision and scheme).
 * LSMC_EINVAL: NULL req or bytes, or an invalid request; LSMC_ENOTIMPL: an
 * unsupported flag combination. */
int lsmc_request_footprint(const lsmc_ctx* ctx, const lsmc_request* req,
                           size_t* bytes);

/* ---- synchronous pricing ----------------------------------------------- */
/* Errors of the pricing calls and plans: LSMC_EINVAL for a NULL pointer or
 * an invalid request (nothing is launched); LSMC_ENOTIMPL for requests of
 * one call that differ in precision, scheme, basis or flags; LSMC_ENOMEM
 * when device memory or the workspace is exhausted; LSMC_ETIMEOUT when a
 * bounded device wait expired (lsmc_set_wait_limit; the context stays
 * usable); LSMC_ECUDA for a failed CUDA call.  The pricing calls run on the
 * context stream and return when the results are in outs. */
/* One contract: price + the Greeks of bumps->greek_mask (Sec. 2.2), its
 * paths simulated by the context's scheme (Sec. 2.2.1) under Philox seed
 * seed; out: host, one result. */
int lsmc_price_greeks(lsmc_ctx* ctx, const lsmc_heston* model,
                      const lsmc_contract* contract, uint32_t n_paths,
                      uint32_t n_steps, int32_t basis, const lsmc_bumps* bumps,
                      uint64_t seed, lsmc_result* out);
/* All strikes of one request, on one path set per scenario (Sec. 2.2.1:
 * the curve fits of every strike read the same paths); outs: host,
 * req->n_strikes results in strike order. */
int lsmc_price_request(lsmc_ctx* ctx, const lsmc_request* req,
                       lsmc_result* outs);
/* A book of requests in one forward and one backward launch (CUDA-graph
 * replayed); outs: host, sum of n_strikes results in request order. */
int lsmc_price_book(lsmc_ctx* ctx, const lsmc_request* reqs, size_t n_reqs,
                    lsmc_result* outs);

/* ---- plans: build once, launch many times ------------------------------ */
/* Validates and expands the requests (scenarios, path groups, job tables),
 * uploads the tables and reserves the device memory (the batching of paths
 * of Sec. 4.1, over all scenarios and requests at once).  *out (host)
 * receives the plan, owned by the caller until lsmc_plan_destroy; errors as
 * for the pricing calls. */
int lsmc_plan_create(lsmc_ctx* ctx, const lsmc_request* reqs, size_t n_reqs,
                     lsmc_plan** out);
/* Enqueues the whole path (forward, backward, Greeks) on the context stream;
 * with use_graph != 0 the sequence is captured once and replayed.
 * Asynchronous.  LSMC_EINVAL for NULL; LSMC_ECUDA if a launch fails. */
int lsmc_plan_launch(lsmc_plan* plan, int32_t use_graph);
/* Waits for the last launch and copies its results to outs (host, the
 * plan's n_results, lsmc_plan_get_info).  LSMC_EINVAL for NULL;
 * LSMC_ETIMEOUT or LSMC_ECUDA as for the pricing calls. */
int lsmc_plan_fetch(lsmc_plan* plan, lsmc_result* outs);
/* Scenario kinds of the bump-and-revalue table (LSMC_SC_*), the index of a
 * revaluation within one result's row of lsmc_plan_fetch_scenarios. */
enum { LSMC_SC_BASE = 0, LSMC_SC_S_UP, LSMC_SC_S_DN, LSMC_SC_SG_UP, LSMC_SC_SG_DN,
       LSMC_SC_V0_UP, LSMC_SC_V0_DN, LSMC_SC_R_UP, LSMC_SC_R_DN, LSMC_SC_T_DN,
       LSMC_SC_T_UP, LSMC_SC_COUNT };
/* The revaluations behind the Greeks of the last launch (Sec. 2.2: the
 * Greeks are differences of these prices): prices (host, n_results x
 * LSMC_SC_COUNT doubles) gets, for result k and scenario kind s, the price of
 * that revaluation at [k * LSMC_SC_COUNT + s], NaN where the request has no
 * such scenario; near_ties (host, optional, same shape) its near-tie
 * decisions (see lsmc_result).  n_results must equal the plan's result
 * count.  Waits for the last launch.  LSMC_EINVAL for a NULL plan or prices
 * or another n_results; LSMC_ECUDA if the copy fails. */
int lsmc_plan_fetch_scenarios(lsmc_plan* plan, double* prices, uint32_t* near_ties,
                              size_t n_results);
/* Device address of the launch's results: *device_ptr (host) receives the
 * address of *count lsmc_result entries, owned by the plan, rewritten by
 * every launch and valid until lsmc_plan_destroy.  LSMC_EINVAL for NULL. */
int lsmc_plan_device_results(lsmc_plan* plan, void** device_ptr, size_t* count);
/* Counters of the plan: kernels per launch, generated and LSMC path-steps,
 * jobs of the backward pass, device bytes held. */
typedef struct lsmc_plan_info {
  uint64_t generated_path_steps, lsmc_path_steps, backward_jobs, device_bytes;
  uint32_t kernels_per_launch, n_results, n_instances, n_groups;
  uint64_t itm_path_steps; /* in-the-money regression path-steps, set by fetch */
  uint64_t h2d_bytes;      /* table bytes uploaded by lsmc_plan_create */
  uint64_t d2h_bytes;      /* bytes read back by each lsmc_plan_fetch */
} lsmc_plan_info;
/* Fills *info (host) with the plan's counters.  LSMC_EINVAL for NULL. */
int lsmc_plan_get_info(const lsmc_plan* plan, lsmc_plan_info* info);
/* The counters of lsmc_plan_get_info that are fixed before any launch, for
 * the plan lsmc_plan_create would build for these requests with backward
 * shape (sub sub-tiles per job, optionally | LSMC_SUB_ITM_HALF; ppt paths
 * per thread of a sub-tile, 0 or a value not compiled for the precision:
 * the precision's default): generated and LSMC
 * path-steps, backward jobs, device bytes, results, instances, path groups
 * and table bytes (h2d_bytes); kernels_per_launch = 4, itm_path_steps =
 * d2h_bytes = 0.  Host only: nothing is allocated and no device is touched;
 * ctx may be NULL (then the library's default precision and scheme).
 * LSMC_EINVAL for a sub-tile count outside 1..64, another bit in sub, ppt
 * not in {0, 2, 4, 8} or an invalid request; LSMC_ENOTIMPL where
 * lsmc_plan_create would give it. */
int lsmc_plan_layout_info(const lsmc_ctx* ctx, const lsmc_request* reqs, size_t n_reqs,
                          uint32_t sub, uint32_t ppt, lsmc_plan_info* info);
/* Per-kernel timing of later launches (CUDA events on the plan's stream,
 * recorded between its kernels; no effect on results).  enable = 0 stops.
 * LSMC_EINVAL for NULL. */
int lsmc_plan_set_timing(lsmc_plan* plan, int32_t enable);
/* Device milliseconds summed over the launches since the previous call:
 * ms[0] setup, ms[1] forward (paths), ms[2] backward (LSMC), ms[3] Greeks
 * (host, 4 doubles); *launches (optional) = number of launches summed.
 * Waits for the last launch.  LSMC_EINVAL for NULL plan or ms; LSMC_ECUDA
 * if an event cannot be read. */
int lsmc_plan_kernel_times(lsmc_plan* plan, double ms[4], uint32_t* launches);
/* Autotuner: times the backward pass of a plan for these requests over its
 * tile shapes -- paths per thread of a sub-tile (2 or 4 for LSMC_FP64 and
 * LSMC_DF, 4 or 8 for LSMC_MIXED) and jobs of 1, 2, 4, ... sub-tiles, each
 * from 2 sub-tiles up also with LSMC_SUB_ITM_HALF where a request has
 * strikes on both sides of S0 (one warm-up and one timed launch each) --,
 * remembers the fastest for later plans of the same precision, basis and
 * size class on this context, and returns it (best_sub, best_ppt, best_ms:
 * optional; best_sub may carry LSMC_SUB_ITM_HALF).  Synchronous on the
 * context stream.  The first failing trial ends the search: the fastest
 * shape timed before it is kept and LSMC_OK returned, else that trial's
 * error (as for lsmc_plan_create and lsmc_plan_fetch). */
int lsmc_autotune(lsmc_ctx* ctx, const lsmc_request* reqs, size_t n_reqs,
                  uint32_t* best_sub, uint32_t* best_ppt, double* best_ms);
/* Frees the plan's device memory once its work is done (stream-ordered).
 * Destroy every plan before the context it was created on.  NULL is
 * ignored. */
void lsmc_plan_destroy(lsmc_plan* plan);

/* Lower and upper bounds of the American price of every strike of one
 * request (the request's bumps are ignored: base scenario only).  The
 * regressions on the request's paths (stream_id) fix an exercise policy
 * (Sec. 2.2.1's Longstaff-Schwartz stage).  Lower bound: that policy applied
 * to independent paths (stream_id ^ 0x80000000, as LSMC_FLAG_OUT_OF_SAMPLE).
 * Upper bound: the dual bound of Andersen and Broadie over the first n_outer
 * of those paths: along each, at every date, n_inner inner paths (Philox
 * counter (j, m, stream_id ^ 0x40000000, 1 + p n_steps + n) for inner path j
 * of outer path p started at date n, step from date m) estimate the value of
 * continuing under the policy; the policy's value process gives a martingale
 * pi, and the bound is the mean of max_n (Z_n - pi_n), Z the payoff
 * discounted to t_0.  Work ~ n_outer n_inner n_steps^2 / 2 path steps.
 * outs: host, n_strikes entries.  LSMC_EINVAL: European style, n_outer = 0
 * or > n_paths, n_inner = 0, more than 16 strikes, n_outer n_steps >= 2^31;
 * LSMC_ENOTIMPL with LSMC_FLAG_REGENERATE.  Synchronous. */
int lsmc_price_bounds(lsmc_ctx* ctx, const lsmc_request* req, uint32_t n_outer,
                      uint32_t n_inner, lsmc_bounds* outs);

/* ---- serving: continuous batching -------------------------------------- */
/* Queues a copy of *req; returns a ticket.  Whenever a slot
 * (config.max_inflight) is free, the oldest pending request and the pending
 * requests right behind it that can share a launch (same precision, scheme
 * and basis; up to config.max_batch, while the workspace bytes of
 * config.hbm_budget allow) are admitted together as one batch: one launch
 * of each kernel, on the slot's own stream, overlapping with the batches
 * already running.  A request is done as soon as its own revaluations are:
 * the backward pass forms its prices and Greeks when its last regression
 * finishes and hands them to the host through page-locked, device-mapped
 * memory, ahead of the rest of its batch (out-of-sample requests finish with
 * their batch).  The backward job size of a request depends on the request
 * alone, so its results are the same whichever batch it runs in, and the
 * same as lsmc_price_request's under the same backward shape.  *ticket
 * (host) receives the ticket.  LSMC_EINVAL or LSMC_ENOTIMPL as for
 * lsmc_request_footprint (nothing is queued); LSMC_ENOMEM when the request
 * alone exceeds the serving workspace; LSMC_EBUSY when the queue
 * (config.queue_capacity) is full; LSMC_ECUDA if the scheduler's streams
 * cannot be created.  (A serving policy: the paper prices one problem at a
 * time.) */
int lsmc_submit(lsmc_ctx* ctx, const lsmc_request* req, uint64_t* ticket);
/* LSMC_PENDING while in flight; LSMC_OK with outs filled (host, n_strikes
 * results; NULL takes the ticket without copying) once done, the ticket then
 * released; the request's own error code if it failed (released too);
 * LSMC_ENOTFOUND for a ticket never issued or already released; LSMC_EINVAL
 * if ctx is NULL. */
int lsmc_poll(lsmc_ctx* ctx, uint64_t ticket, lsmc_result* outs);
/* Blocks up to timeout_s (< 0: no limit) for the ticket, then as lsmc_poll
 * (LSMC_PENDING if the time ran out first). */
int lsmc_wait(lsmc_ctx* ctx, uint64_t ticket, lsmc_result* outs,
              double timeout_s);
/* Per-ticket timing (seconds since lsmc_create, host steady clock): submit,
 * admission to the device and completion (each output optional, host).
 * Also answers for released tickets (the last 2^20 are remembered).
 * LSMC_ENOTFOUND for other tickets; LSMC_EINVAL if ctx is NULL. */
int lsmc_ticket_times(lsmc_ctx* ctx, uint64_t ticket, double* submit_s,
                      double* admit_s, double* done_s);

/* ---- measurement ---------------------------------------------------------- */
/* Measured throughput of the arithmetic pipes that bound this library's
 * kernels, the denominators of their roofline fractions (a measurement aid;
 * the paper has no counterpart).  fp64_tflops and fp32_tflops: fused
 * multiply-adds in double and in float (2 flops each); xu_tops: the
 * special-function unit (base-2 exponentials, one operation each).  Each
 * probe runs 8 independent dependency chains per thread on 8 CTAs of 256
 * threads per SM, 10 to 20 ms per launch; the fastest of five launches
 * after two warm-up launches counts (CUDA events); *_ms are those times.  Synchronous on an internal stream of the
 * device; changes no device setting and allocates nothing.  LSMC_EINVAL for a
 * bad device ordinal or NULL out, LSMC_ENODEV without a device. */
typedef struct lsmc_peaks {
  double fp64_tflops, fp32_tflops, xu_tops;
  double fp64_ms, fp32_ms, xu_ms;
  int32_t sms;
  int32_t reserved;
} lsmc_peaks;
int lsmc_measure_peaks(int32_t device, lsmc_peaks* out);

/* The checked build's bounds report (a diagnostic; the paper has none).  A
 * build of this library compiled with LSMC_CHECKED tests every global-memory
 * access of its kernels against the byte ranges the launch owns (the plan's
 * allocation, the caller's arrays of a stage call); an access outside them
 * is skipped and the first one is recorded.  *code: 0, or 3 once an access
 * fell outside; *line: the kernel source line of that access.  reset != 0
 * clears the record.  Synchronises the current device.  The ordinary build
 * returns LSMC_ENOTIMPL; LSMC_EINVAL for NULL pointers. */
int lsmc_check_report(uint32_t* code, uint32_t* line, int32_t reset);

/* ---- stage entry points (device pointers; for parity tests) ------------- */
/* Philox4x32-10 of n counters: d_ctr n x 4 uint32 (device), key = (key_lo,
 * key_hi); d_out n x 4 uint32 (device).  (Random inputs of Sec. 2.2.1.)
 * Asynchronous on cuda_stream (NULL: the default stream); LSMC_EINVAL for
 * NULL arrays with n > 0, LSMC_ECUDA if the launch fails. */
int lsmc_philox(const uint32_t* d_ctr, uint32_t key_lo, uint32_t key_hi,
                uint32_t* d_out, size_t n, void* cuda_stream);
/* Random inputs of n (path, step) pairs under (seed, stream_id), the two
 * per path and step of Sec. 2.2.1: d_path, d_step (device, n uint32 each);
 * d_out (device) is n x 3 (U_V, Z_V, Z_X) as double (LSMC_FP64: 52-bit
 * grid), float (LSMC_MIXED: 23-bit grid) or float pairs (LSMC_DF: the FP64
 * values split).  Asynchronous on cuda_stream; LSMC_EINVAL for NULL arrays
 * with n > 0 or an unknown precision, LSMC_ECUDA if the launch fails. */
int lsmc_draws(uint64_t seed, uint32_t stream_id, const uint32_t* d_path,
               const uint32_t* d_step, size_t n, int32_t precision,
               void* d_out, void* cuda_stream);
/* The exponential step of the path generation (Sec. 2.2.1: the stored S is
 * S0 exp(x) of the log price x) on n values: d_x, d_y (device) of the
 * precision (double, float, or float pairs hi, lo).  In double, Tang's
 * table-driven method for |x| < 512 (within one unit in the last place) and
 * CUDA's exp beyond; float pairs by a Cody-Waite reduction and a 128-entry
 * table (within 2e-14 relative for |x| <= 70, where the result's low word
 * stays a normal float); single precision by CUDA's __expf.  Asynchronous on cuda_stream;
 * LSMC_EINVAL for NULL arrays (n > 0) or an unknown precision. */
int lsmc_exp(const void* d_x, void* d_y, size_t n, int32_t precision, void* cuda_stream);
/* The Gaussian transform of the random inputs (Sec. 2.2.1: the normal draws
 * of the Heston step from uniforms) on n uniforms: d_u, d_z (device) double
 * (LSMC_FP64) or float (LSMC_MIXED); z = Phi^-1(u) with 1 - u formed in the
 * precision, exact for u on its uniform grid (the points (m + 1/2) 2^-52,
 * (m + 1/2) 2^-23 that lsmc_draws uses).  Double: w = -log(4 u (1 - u)) by
 * a table-driven logarithm and polynomials in w or sqrt(w) (Giles'
 * transformation, own fit), within 6e-16 of Phi^-1(u), max(1, |z|)
 * relative; float: within 1e-6.  Asynchronous on cuda_stream; LSMC_EINVAL for
 * NULL arrays (n > 0) or an unknown precision, LSMC_ENOTIMPL for LSMC_DF
 * (its quantile reads the random words: lsmc_draws). */
int lsmc_quantile(const void* d_u, void* d_z, size_t n, int32_t precision, void* cuda_stream);

/* Heston paths (Sec. 2.2.1: variance, log price, exponential; the
 * step-major layout of Sec. 4.1):
 * d_S, d_V (device) are (n_steps + 1) x n_paths, step-major, double, float
 * or float pairs by precision; row 0 holds S0 and v0.  V holds max(v, 0) under
 * FT_EULER.  Path p, step n draws Philox counter (p, n, stream_id, 0) under
 * key seed.  Asynchronous on cuda_stream (its small tables are allocated
 * and freed stream-ordered); LSMC_EINVAL for NULL pointers or invalid model
 * parameters, LSMC_ENOMEM, LSMC_ECUDA. */
int lsmc_paths(const lsmc_heston* model, double T, int32_t scheme,
               int32_t precision, uint32_t n_paths, uint32_t n_steps,
               uint64_t seed, uint32_t stream_id, void* d_S, void* d_V,
               void* cuda_stream);
/* STAC-A2 path reduction (Sec. 2.2.1 and Sec. 4.1: Heston QE paths of every
 * asset, their exponential, and the Longstaff-Schwartz path reduction that
 * keeps, for every path and date, the largest value held by any asset).
 * models: host, n_assets (1..64) Heston models, one per asset; element
 * (path, asset, date) draws from Philox counter (path, date, stream_id,
 * asset) under key seed.  rho_assets in [0, 1]: equicorrelation of the
 * assets' log-price shocks through one common factor per (path, date)
 * (counter (path, date, stream_id, 0xFFFFFFFF)); 0 = independent assets,
 * two random numbers per element as in the paper.  d_M (device): (n_steps
 * + 1) x n_paths values of the precision (double, float, or float pairs hi,
 * lo), row n = date n, row 0 = the largest S0.  Asynchronous on cuda_stream;
 * LSMC_EINVAL before any launch for invalid arguments. */
int lsmc_multi_asset_max(const lsmc_heston* models, uint32_t n_assets, double T,
                         int32_t scheme, int32_t precision, double rho_assets,
                         uint32_t n_paths, uint32_t n_steps, uint64_t seed,
                         uint32_t stream_id, void* d_M, void* cuda_stream);

/* Longstaff-Schwartz backward pass over given paths (Sec. 2.2.1: the
 * reduction and the least-squares curve fit of every exercise date; same
 * layout as lsmc_paths output).  d_out (device, 5 doubles): price, price_se,
 * european_price, continuation value, near-tie decisions (see lsmc_result).  d_beta (device, optional):
 * n_steps x 6 doubles, row n = coefficients at date n (NaN if none).
 * d_n_singular (device, optional): 1 uint32.  Returns after the work has
 * finished (waits on cuda_stream).  LSMC_EINVAL for NULL d_S, model,
 * contract or d_out, NULL d_V with LSMC_BASIS_SV2, or invalid parameters;
 * LSMC_ENOMEM; LSMC_ETIMEOUT when a bounded device wait expired;
 * LSMC_ECUDA. */
int lsmc_backward(const void* d_S, const void* d_V, uint32_t n_paths,
                  uint32_t n_steps, int32_t precision, const lsmc_heston* model,
                  const lsmc_contract* contract, int32_t basis, double* d_out,
                  double* d_beta, uint32_t* d_n_singular, void* cuda_stream);

/* The backward pass of lsmc_backward for callers that cannot allocate device
 * memory (another allocator owns the device, cudaMalloc/cudaFree would
 * synchronise a latency-critical path, or the device is nearly full).  The
 * paper has no counterpart; this is a deployment variant.  Same arguments,
 * layouts and results as lsmc_backward; it calls no cudaMalloc, cudaFree or
 * other allocating routine.  Its scratch is a 16 MiB array that the library
 * keeps in device memory on every device that loads it, until the process
 * exits; a request needing more (about n_paths x 8 bytes plus n_steps x 64
 * bytes in FP64) returns LSMC_ENOMEM before anything is launched.  The
 * first call on a device, and the first after the device's context changes
 * (cudaDeviceReset, or a caller's own driver context), looks up the array's
 * device address (do that call before any stream capture).  All calls
 * share the one array and leave their contents in it: calls whose work
 * overlaps on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  Returns after the work has finished, on success
 * and on failure alike (the call waits on cuda_stream). */
int lsmc_backward_noalloc(const void* d_S, const void* d_V, uint32_t n_paths,
                          uint32_t n_steps, int32_t precision,
                          const lsmc_heston* model, const lsmc_contract* contract,
                          int32_t basis, double* d_out, double* d_beta,
                          uint32_t* d_n_singular, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
