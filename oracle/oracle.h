/*
 * oracle.h -- plain FP64 CPU oracle for the Heston / Longstaff-Schwartz /
 * bump-and-revalue Greeks path of "Low-power option Greeks" (Klaisoongnoen,
 * Brown, Thomson Brown, HEART '22).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this code; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no header, table or
 * helper with the CUDA path.
 *
 * Every function follows the definition of the step it implements, in the
 * order the method states it, in double precision, compiled without FMA
 * contraction.  The paper itself prints no formulas: it names the method
 * (Heston model, Andersen quadratic-exponential discretisation, two
 * double-precision random inputs per path/asset/step, exponential of the log
 * price, Longstaff-Schwartz regression with a quadratic curve fit; Sec. 2.2
 * and Sec. 2.2.1) and cites the original papers for the formulas.  The
 * readings taken where it is silent are listed per function below.
 *
 * Pins (tests/test_oracle_*.py): Philox against the cuRAND host generator;
 * the normal quantile against scipy's ndtri; the QE variance step against its
 * exact first two conditional moments; the FT-Euler step against its xi = 0
 * closed form; path prices against the Heston characteristic-function price
 * and Black-Scholes; the backward induction against a least-squares solve by
 * QR on tiny path sets and against a stopping-time reconstruction; American
 * prices against a CRR tree restricted to the same exercise dates; Greeks
 * against Black-Scholes Greeks; the multi-asset reduction against the
 * single-asset paths and the distribution of the maximum of (correlated)
 * lognormals in the Black-Scholes limit; the
 * out-of-sample estimator against the in-sample one on the same paths and
 * the binomial Bermudan price; the 16-bit rounding against numpy's float16
 * and torch's bfloat16 conversions and the European Lipschitz bound; the
 * dual upper bound against the immediate-exercise floor, the martingale's
 * zero mean and the binomial bracket.  No function here is unpinned.
 */
#ifndef LSMC_ORACLE_H
#define LSMC_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PUT = 0, ORC_CALL = 1 };
enum { ORC_AMERICAN = 0, ORC_EUROPEAN = 1 };
enum { ORC_QE = 0, ORC_FT_EULER = 1 };
enum { ORC_BASIS_S2 = 0, ORC_BASIS_SV2 = 1 };
/* uniform grid: 52-bit (double) or 23-bit (single-precision) mantissa */
enum { ORC_GRID_F64 = 0, ORC_GRID_F32 = 1 };
enum { ORC_GREEK_DELTA = 1, ORC_GREEK_GAMMA = 2, ORC_GREEK_VEGA = 4,
       ORC_GREEK_RHO = 8, ORC_GREEK_THETA = 16 };
/* scenario kinds, in the order scenarios are laid out */
enum { ORC_SC_BASE = 0, ORC_SC_S_UP, ORC_SC_S_DN, ORC_SC_SG_UP, ORC_SC_SG_DN,
       ORC_SC_V_UP, ORC_SC_V_DN, ORC_SC_R_UP, ORC_SC_R_DN, ORC_SC_T_DN,
       ORC_SC_T_UP, ORC_SC_COUNT };

typedef struct {
  double S0, r, q, v0, kappa, theta, xi, rho;
} orc_heston;

typedef struct {
  double rel_dS, rel_dS_gamma, rel_dv0, abs_dr, abs_dT;
  uint32_t greek_mask;
  uint32_t pad_;
} orc_bumps;

typedef struct {
  double price, price_se, delta, gamma, vega, rho, theta, european_price;
  uint32_t n_singular, n_revaluations;
  int32_t status;
  int32_t pad_;
} orc_result;

/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds on a 128-bit counter
 * under a 64-bit key. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);

/* The uniforms behind the random inputs of Sec. 2.2.1 (the paper leaves
 * their grid open; this one is symmetric, so 1 - u is exact and the
 * quantile is odd about 1/2): (m + 1/2) 2^-52 with m = the top 52 bits of
 * (hi:lo); never 0 or 1. */
double orc_uniform_f64(uint32_t hi, uint32_t lo);
/* The same in single precision: (m + 1/2) 2^-23 with m = the top 23 bits
 * of w; never 0 or 1. */
double orc_uniform_f32(uint32_t w);

/* Standard normal quantile, the map from uniforms to the normal draws of
 * Sec. 2.2.1, by its definition: the root z of (1/2) erfc(-z / sqrt 2) = u
 * (bracketed Newton iteration). */
double orc_norm_inv(double u);

/* The random inputs of one path step (Sec. 2.2.1: two random numbers per
 * path, asset and time step): Philox of counter
 * (path, step, stream, 0) under key (seed lo, seed hi) gives (U_V, Z_V, Z_X),
 * Z = quantile(U).  out = {U_V, Z_V, Z_X}. */
void orc_draws(uint64_t seed, uint32_t stream, uint32_t path, uint32_t step,
               int grid, double out[3]);

/* orc_draws for asset `asset` of a multi-asset path (the STAC-A2 form of
 * Sec. 2.2.1): counter (path, step, stream, asset); orc_draws is asset 0. */
void orc_draws_asset(uint64_t seed, uint32_t stream, uint32_t path, uint32_t step,
                     uint32_t asset, int grid, double out[3]);

/* Andersen QE step: out = {x1, v1}. */
void orc_qe_step(const orc_heston* m, double dt, double x, double v,
                 double uV, double zV, double zX, double out[2]);
/* Full-truncation Euler step (Lord, Koekkoek and van Dijk, 2010: v+ =
 * max(v, 0) in drift and diffusion), offered beside the paper's QE scheme
 * (Sec. 2.2.1): out = {x1, v1 (raw), max(v1, 0)}. */
void orc_ft_step(const orc_heston* m, double dt, double x, double v,
                 double zV, double zX, double out[3]);

/* Heston paths in the order of Sec. 2.2.1 (per step the variance, then the
 * log price, then its exponential), stored step-major as in Sec. 4.1: path
 * matrices S[n*P + p], V[n*P + p] for n = 0..N (row 0 = S0, v0). */
int orc_paths(const orc_heston* m, double T, int scheme, int grid,
              uint32_t P, uint32_t N, uint64_t seed, uint32_t stream,
              double* S, double* V, int n_threads);

/* One path (index `path`) of orc_paths (Sec. 2.2.1), simulated alone:
 * S[n], V[n] for n = 0..N. */
int orc_path_one(const orc_heston* m, double T, int scheme, int grid,
                 uint32_t path, uint32_t N, uint64_t seed, uint32_t stream,
                 double* S, double* V);

/* STAC-A2 path reduction (Sec. 2.2.1, Sec. 4.1): A Heston assets per path,
 * asset a with model models[a]; M[n*P + p] = max over assets of S_a at date
 * n (n = 0..N).  Element (path, asset, date) draws from Philox counter
 * (path, date, stream, asset).  With rho_assets > 0 the log-price shocks of
 * the assets share one factor (equicorrelation rho_assets):
 * Z_X,a <- sqrt(rho_assets) Z_c + sqrt(1 - rho_assets) Z_X,a, with Z_c the
 * quantile of the words (2, 3) grid point of counter
 * (path, date, stream, 0xFFFFFFFF).  rho_assets = 0: independent assets,
 * two random numbers per element as in the paper.  Returns 0 or < 0. */
int orc_multi_max(const orc_heston* models, uint32_t A, double T, int scheme, int grid,
                  double rho_assets, uint32_t P, uint32_t N, uint64_t seed,
                  uint32_t stream, double* M, int n_threads);
/* The path of one asset of one multi-asset path (Sec. 2.2.1; same
 * arithmetic as orc_multi_max): S[n] for n = 0..N. */
int orc_asset_path(const orc_heston* m, uint32_t asset, double T, int scheme, int grid,
                   double rho_assets, uint32_t path, uint32_t N, uint64_t seed,
                   uint32_t stream, double* S);

/* Longstaff-Schwartz backward induction over given paths.
 * out = {price, price_se, european_price, continuation}.
 * beta (optional): N*6 doubles, row n holds the step-n coefficients (NaN if
 * no regression at n).  exercise (optional): N*P bytes, 1 where path p
 * exercises at step n.  Returns 0 or a negative error. */
int orc_lsmc(const double* S, const double* V, uint32_t P, uint32_t N,
             double S0, double K, double T, double r, double theta, int type,
             int style, int basis, double out[4], uint32_t* n_singular,
             double* beta, uint8_t* exercise);

/* Near ties and reversed decisions (a test hook; without it the functions
 * are the plain method).  An exercise decision, payoff h against fitted
 * continuation value c at the decision's date, is a near tie when
 * |h - c| <= tie_rel max(|c|, h): another correct rounding of the same
 * arithmetic may take it the other way, so a result computed with other
 * roundings is correct when it equals this oracle's under some set of its
 * near-tie decisions reversed.  Keys: n P + p for the decision of path p at
 * date n in the regressions' pass, ORC_KEY_PRICING | (n P + p) in the
 * pricing pass of the out-of-sample estimator.  ties (optional) receives up
 * to max_ties keys of the near ties met, n_ties counts them all; flips
 * (sorted ascending) lists the decisions to take the other way. */
#define ORC_KEY_PRICING (1ull << 62)
#define ORC_MAX_ALT_KEYS 12
typedef struct {
  double tie_rel;       /* < 0: no near-tie report */
  uint64_t* ties;
  uint32_t max_ties;
  uint32_t n_ties;
  const uint64_t* flips;
  uint32_t n_flips;
} orc_tie_ctl;

/* orc_lsmc (Sec. 2.2.1's Longstaff-Schwartz stage) under a tie control
 * (ctl may be NULL: then it is orc_lsmc). */
int orc_lsmc_tie(const double* S, const double* V, uint32_t P, uint32_t N,
                 double S0, double K, double T, double r, double theta, int type,
                 int style, int basis, double out[4], uint32_t* n_singular,
                 orc_tie_ctl* ctl);

/* Out-of-sample Longstaff-Schwartz: the exercise policy of the regressions on
 * paths (SA, VA) applied to the independent paths (SB, VB) of the same model
 * (first date in 1..N-1 where an in-the-money path's payoff beats the fitted
 * continuation value, else N).  out = {price, price_se, european price on
 * B, mean discounted cash flow}.  With SB = SA, VB = VA it is orc_lsmc. */
int orc_lsmc_oos(const double* SA, const double* VA, const double* SB, const double* VB,
                 uint32_t P, uint32_t N, double S0, double K, double T, double r,
                 double theta, int type, int style, int basis, double out[4],
                 uint32_t* n_singular);

/* Scenario table of a bump specification (the Greeks that Sec. 2.2 names
 * as the purpose of the run, with no method: here central bump-and-revalue
 * differences under common random numbers): fills up to ORC_SC_COUNT models,
 * maturities and kinds; returns the number of scenarios or a negative error. */
int orc_scenarios(const orc_heston* m, double T, const orc_bumps* b,
                  orc_heston* models, double* Ts, int* kinds);

/* Price and Greeks (Sec. 2.2) of n_strikes contracts sharing one path set
 * per scenario (Sec. 2.2.1: paths, then the Longstaff-Schwartz stage).
 * scen_prices (optional): n_scen * n_strikes scenario values. */
int orc_price_greeks(const orc_heston* m, int type, int style, double T,
                     const double* strikes, uint32_t n_strikes, uint32_t P,
                     uint32_t N, int scheme, int grid, int basis,
                     const orc_bumps* b, uint64_t seed, uint32_t stream,
                     int n_threads, orc_result* out, double* scen_prices);

/* orc_price_greeks (Sec. 2.2) with the path store kept in double (store 0)
 * or rounded to 16 bits (store 1: binary16, 2: bfloat16; the storage
 * analogue of the data-type study of Sec. 4.2) and, with out_of_sample != 0,
 * every scenario's price the
 * out-of-sample estimate, regressions on stream `stream`, pricing paths on
 * stream `stream ^ 0x80000000`. */
int orc_price_greeks_ex(const orc_heston* m, int type, int style, double T,
                        const double* strikes, uint32_t n_strikes, uint32_t P,
                        uint32_t N, int scheme, int grid, int basis,
                        const orc_bumps* b, uint64_t seed, uint32_t stream,
                        int out_of_sample, int store, int n_threads, orc_result* out,
                        double* scen_prices);

/* The Greeks of one strike (Sec. 2.2; central differences of the
 * revaluations) from its revaluations: vals[s] is the price of
 * scenario s of the table orc_scenarios gives (kinds[s] its kind, n_sc
 * scenarios).  Fills price, the Greeks of b->greek_mask (NaN otherwise) and
 * n_revaluations; price_se and european_price are NaN. */
void orc_greeks_from_values(const orc_heston* m, const orc_bumps* b, const int* kinds,
                            const double* vals, int n_sc, orc_result* out);

/* One revaluation (Sec. 2.2.1's Longstaff-Schwartz price of one scenario)
 * of orc_price_greeks_ex (scenario index sc of the table,
 * strike K) under reversed decisions: out[i] (2^n_keys values) is its price
 * with the decisions whose bit is set in i reversed, bit j standing for the
 * j-th smallest of the n_keys (<= ORC_MAX_ALT_KEYS) keys.  n_ties (optional):
 * the plain run's near ties at tie_rel are counted there and their keys
 * written to ties (up to max_ties).  Returns 0 or < 0. */
int orc_scenario_alternatives(const orc_heston* m, int type, int style, double T, double K,
                              uint32_t P, uint32_t N, int scheme, int grid, int basis,
                              const orc_bumps* b, uint64_t seed, uint32_t stream,
                              int out_of_sample, int store, int sc, double tie_rel,
                              const uint64_t* keys, uint32_t n_keys, double* out,
                              uint64_t* ties, uint32_t max_ties, uint32_t* n_ties,
                              int n_threads);

/* Dual (Andersen-Broadie) upper bound of the American price for each strike,
 * with the exercise policy fitted on the P paths of `stream` (in-sample
 * regressions).  out[k*6 + 0..5]: lower bound (out-of-sample estimator on the
 * P pricing paths of stream ^ 0x80000000) and its standard error, upper
 * bound (mean over the first n_outer pricing paths of max_n (Z_n - pi_n))
 * and its standard error, the mean of the martingale at maturity pi_N and
 * its standard error (zero in expectation).  Inner path j of outer path p
 * started at date n draws from counter (j, m, stream ^ 0x40000000,
 * 1 + p N + n) for its step from date m.  Returns 0 or < 0. */
int orc_dual_bound(const orc_heston* m, int type, double T, const double* strikes,
                   uint32_t n_strikes, uint32_t P, uint32_t N, int scheme, int grid, int basis,
                   uint64_t seed, uint32_t stream, uint32_t n_outer, uint32_t n_inner,
                   int n_threads, double* out);

/* The 16-bit storage of the data-type study (Sec. 4.2, Table 4): rounding
 * to nearest, ties to even, from a double to IEEE binary16 (orc_round_f16)
 * and to bfloat16 (orc_round_bf16), returned as doubles; overflow gives
 * infinity. */
double orc_round_f16(double x);
double orc_round_bf16(double x);
/* y[i] = x[i] rounded as above (store 1: binary16, 2: bfloat16). */
void orc_round_n(const double* x, double* y, size_t n, int store);

/* Array forms of orc_philox4x32_10, orc_norm_inv and orc_draws (Sec. 2.2.1's
 * random inputs; plain loops over the scalar functions). */
void orc_philox_n(const uint32_t* ctr, const uint32_t key[2], uint32_t* out,
                  size_t n);
void orc_norm_inv_n(const double* u, double* z, size_t n);
void orc_draws_n(uint64_t seed, uint32_t stream, const uint32_t* path,
                 const uint32_t* step, size_t n, int grid, double* out);

#ifdef __cplusplus
}
#endif
#endif
