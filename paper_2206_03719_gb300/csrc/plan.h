// plan.h -- device-side tables of one launch (host planner <-> kernels).
//
// A launch prices a set of "contracts" (a request = one model, one maturity,
// several strikes).  Each contract's bump scenarios are folded onto "path
// groups": scenarios whose paths are the same simulation.  Scenarios that
// only move S0 share x = ln(S/S0) exactly; scenarios that only move r share
// the variance path and shift x by n (dr) dt, i.e. scale S by exp(n dr dt).
// v0 and T bumps need their own simulation.  A regression "instance" is one
// (scenario, strike) pair; it reads its group's stored exp(x) and v rows.
#pragma once

#include <cstdint>

namespace lsmc {

constexpr int kBlock = 256;      // threads per CTA of the backward pass
constexpr int kOosTile = 1024;   // paths per CTA of the out-of-sample pricing pass
constexpr int kOosConsts = 12;   // per-date constants of the out-of-sample pricing pass
constexpr int kScreenBytes = 48; // one float screen of an exercise test (12 floats)
constexpr int kFwdBlock = 128;   // threads (paths) per CTA of the forward pass
constexpr int kMaxGroups = 5;    // path groups per contract (base, v0+, v0-, T-, T+)
constexpr int kNSum = 25;        // doubles per tile partial
// partial layout: 15 monomials x^a w^b (a + b <= 4), 6 right-hand sides,
// European payoff sum, sum of Y, sum of Y^2, near-tie count
constexpr int kSlotRhs = 15;
constexpr int kSlotEuro = 21;
constexpr int kSlotSumY = 22;
constexpr int kSlotSumY2 = 23;
constexpr int kSlotTies = 24;
// an exercise decision whose discounted payoff lies within this relative
// distance of the fitted continuation value is counted as a near tie: two
// correct implementations that round differently may decide it differently
constexpr double kTieRel = 1e-10;

enum : int32_t { kSchemeQE = 0, kSchemeFT = 1 };
// precisions (values of lsmc_request.precision)
enum : int32_t { kPrecFP64 = 0, kPrecMixed = 1, kPrecDF = 2 };
enum : int32_t { kPut = 0, kCall = 1 };
enum : int32_t { kAmerican = 0, kEuropean = 1 };
enum : int32_t { kBasisS2 = 0, kBasisSV2 = 1 };
// element type of the path store (E and V rows): the working precision,
// IEEE binary16 or bfloat16
enum : int32_t { kStoreNative = 0, kStoreF16 = 1, kStoreBF16 = 2 };

// error codes written by kernels into Control::error
enum : uint32_t { kDevErrTimeout = 1, kDevErrBadJob = 2, kDevErrBadIndex = 3 };

// Checked build (compiled with LSMC_CHECKED): the byte ranges a launch may
// touch.  Every global-memory access of the kernels is tested against them
// (checked.cuh); one that falls outside every range is skipped (a load gives
// zero), and the first such access records kDevErrBadIndex in *err and its
// source line in *info.  The ordinary build carries none of this.
constexpr int kMaxRanges = 8;
struct CheckRanges {
  unsigned long long lo[kMaxRanges], hi[kMaxRanges];  // [lo, hi)
  uint32_t n;
  uint32_t* err;
  uint32_t* info;
};
// an extra parameter (and its argument) of the kernels and launchers that
// take no argument structure, in the checked build only
#ifdef LSMC_CHECKED
#define CHK_PARAM , ::lsmc::CheckRanges chk
#define CHK_ARG(x) , (x)
#else
#define CHK_PARAM
#define CHK_ARG(x)
#endif

// ---- forward ------------------------------------------------------------
struct FwdGroup {
  double v0, kappa, theta, xi, rho, r, q, dt;
  double out_scale;   // E row value = out_scale * exp(x)
  void* E;            // rows of dates row0.., ld elements apart (FwdArgs::row0)
  void* V;            // the same for v (nullptr: not stored)
  void* E_row0;       // optional row 0 (= out_scale)
  void* V_row0;       // optional row 0 (= v0)
  void* CX;           // regenerate mode: saved x at dates k ck_stride (index k)
  void* CV;           // regenerate mode: saved v (raw) at the same dates
  uint64_t ld;
};

struct FwdContract {
  uint64_t seed;
  uint32_t stream_id;
  uint32_t P, N;
  uint32_t group0, n_groups;
  uint32_t block0;    // first CTA of this contract in the grid
};

struct FwdArgs {
  const FwdContract* contracts;
  const FwdGroup* groups;
  uint32_t n_contracts;
  uint32_t n_blocks;
  // dates simulated: (n0, n1] from the state at n0 (n0 = 0: the initial
  // state, else the saved state at n0); n1 = 0 means each contract's N
  uint32_t n0, n1;
  uint32_t row0;        // date of E/V row index 0 (1: rows of dates 1..N)
  uint32_t ck_stride;   // regenerate mode: dates between saved states (else 0)
  int32_t store_rows;   // write the E/V rows
  int32_t save_states;  // save the state at every date k ck_stride < N
  unsigned long long* next_job;  // if set, block 0 stores next_job_value there
  unsigned long long next_job_value;
  uint32_t stream_xor;  // xored into every contract's stream id (pricing paths)
  int32_t store_fmt;    // element type of the E/V rows (kStore*)
  // every contract of the launch draws under one key: its Philox round keys
  // (key advanced r times at 2r, 2r + 1); uniform_key = 0 otherwise
  int32_t uniform_key;
  uint32_t rk[20];
#ifdef LSMC_CHECKED
  CheckRanges chk;
#endif
};

// ---- STAC-A2 multi-asset path reduction --------------------------------------
constexpr int kMaxAssets = 64;
struct MultiModel {       // one asset's Heston model
  double S0, r, q, v0, kappa, theta, xi, rho;
};
struct MultiArgs {        // passed by value (about 4 KB of kernel parameters)
  MultiModel assets[kMaxAssets];
  uint32_t n_assets, P, N, stream_id;
  uint64_t seed;
  double T;
  double sqrt_rho, sqrt_1m_rho;  // loadings of the common shock (0, 1: independent)
  void* M;                       // (N + 1) x P values of the working precision
#ifdef LSMC_CHECKED
  CheckRanges chk;
#endif
};

// ---- Greeks ---------------------------------------------------------------
// device mirror of lsmc_result (same layout; checked in capi.cpp)
struct DevResult {
  double price, price_se, delta, gamma, vega, rho, theta, european_price;
  uint32_t n_singular_solves, n_revaluations;
  int32_t status;
  uint32_t n_near_ties;
};

struct GreekOut {
  int32_t res[11];     // result slot per scenario kind (-1 absent)
  uint32_t mask;
  double S0, v0, hS, hG, hV, dR, dT;
};

// scenario kinds (layout order)
enum : int32_t { kScBase = 0, kScSUp, kScSDn, kScSgUp, kScSgDn, kScVUp, kScVDn,
                 kScRUp, kScRDn, kScTDn, kScTUp, kScCount };

// ---- backward -------------------------------------------------------------
struct BwdInstance {
  const void* E;      // group rows 1..N (exp(x) scaled by the group's out_scale)
  const void* V;      // group variance rows 1..N (nullptr for basis S2)
  uint64_t ld;
  void* Y;            // P cash flows discounted to t_0 (owned by this instance)
  double* partial;    // tiles x kNSum
  double* beta_hist;  // optional N x 6
  double* scale_tab;  // 2 (N + 1): S multipliers of E, then discount factors
                      // exp(-r n dt) (filled by the setup kernel)
  double spot;        // scenario S0 (exercise value at t_0)
  double scale0;      // S0 multiplier of E rows
  double dr_dt;       // S multiplier exp(n dr_dt) (folded rate bump)
  double r, dt, T, K, theta;
  double disc, disc_T, invK, inv_theta, h0;   // filled by the setup kernel
  uint32_t P, N, tiles, gens;
  int32_t type, style, basis;
  uint32_t out_index; // result slot
  uint32_t sub;       // sub-tiles of kBlock * PPT paths per job (a tile)
  uint32_t req;       // the instance's request (contract) in the launch
  uint32_t pad_;
  double* beta_z;     // out of sample: N x 8, date n: 6 coefficients (cash flows
                      // discounted to t_0), then 1 if the regression was solved
  double* oos_sum;    // out of sample: per pricing tile of kOosTile paths: sum Z,
                      // sum Z^2, European sum, near ties
  void* oos_tab;      // out of sample: (N + 1) x kOosConsts values of the working
                      // precision per date: 6 coefficients, solved flag, S multiplier,
                      // discount factor as a pair (hi, lo), in-the-money threshold
  void* oos_screen;   // out of sample: (N + 1) float screens of the exercise test
                      // (ScreenConsts, kScreenBytes each)
};

struct BwdState {
  uint32_t arrive;    // tile arrivals, all generations
  uint32_t ready;     // generations solved and published
  uint32_t singular;
  uint32_t beta_ok;
  double beta[6];
  double euro_sum;
  double itm;         // in-the-money path-steps seen by the regressions
  double ties;        // near-tie exercise decisions
};

struct BwdResult {
  double price, se, euro, cont, ties, itm;
  uint32_t singular;
  uint32_t done;
};

struct Control {
  unsigned long long next_job;
  uint32_t error;
  uint32_t error_info;
};

struct BwdArgs {
  const BwdInstance* inst;   // sorted by gens, descending
  BwdState* state;
  BwdResult* results;        // indexed by BwdInstance::out_index
  const unsigned long long* round_off;  // n_rounds + 1
  const uint32_t* cum_tiles; // n_inst + 1 (over the sorted instances)
  const uint32_t* active;    // instances active in each round
  Control* ctl;
  unsigned long long total_jobs;
  unsigned long long timeout_ns;
  uint32_t n_rounds, n_inst;
  uint32_t row0;             // date of E/V row index 0 of the instances' rows
  int32_t store_fmt;         // element type of the E/V rows (kStore*)
  // Per-request completion (serving): the last instance of a request to
  // finish forms the request's price and Greeks and hands them to the host
  // at once, ahead of the rest of the launch; flag_host == nullptr: off.
  uint32_t* req_count;       // per request: instances finished (zeroed with the state)
  const uint32_t* req_info;  // per request: instances, first GreekOut, GreekOuts
  const GreekOut* greeks;
  DevResult* out_host;       // host-mapped: a DevResult per GreekOut
  uint32_t* flag_host;       // host-mapped: per request, 1 once its results are there
#ifdef LSMC_CHECKED
  CheckRanges chk;
#endif
};

// ---- dual upper bound ------------------------------------------------------
constexpr int kMaxDualStrikes = 16;  // strikes of one request in the dual pass
constexpr int kDualOut = 8;          // doubles of output per strike
struct DualArgs {
  const BwdInstance* inst;           // the plan's instances (policy tables oos_tab)
  uint32_t inst_of_strike[kMaxDualStrikes];
  FwdGroup group;                    // the base simulation's model
  uint64_t seed;
  uint32_t stream;                   // the request's stream id
  int32_t type;
  uint32_t N, n_outer, n_inner, n_strikes;
  void* X;                           // (N + 1) x n_outer outer log prices (working precision)
  void* V;                           // the same for the variance (state)
  double* Q;                         // n_strikes x n_outer x N inner estimates
  double* dmax;                      // n_strikes x n_outer pathwise maxima
  double* piN;                       // n_strikes x n_outer martingale at maturity
  uint32_t* inner_ties;              // n_outer x N near ties of the inner rules
  uint32_t* max_ties;                // n_strikes x n_outer near ties along the outer paths
  double* out;                       // n_strikes x kDualOut: bound, its standard error,
                                     // mean pi_N, its standard error, near ties
#ifdef LSMC_CHECKED
  CheckRanges chk;
#endif
};

}  // namespace lsmc
