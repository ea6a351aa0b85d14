// backward.cu -- Longstaff-Schwartz backward induction, estimator and Greeks.
//
// The paper's Longstaff-Schwartz stage is a reduction followed by a
// quadratic curve fit per exercise date (Sec. 2.2.1); here the fit is a
// least-squares regression of the discounted cash flow on a scaled basis over
// the in-the-money paths, solved from its normal equations.
//
// Work decomposition.  A regression instance (scenario x strike) has one job
// per (exercise date, path tile).  Jobs are numbered round-major (round r =
// the r-th date counted back from maturity) and CTAs of a persistent grid take
// them from one atomic counter, so no co-residency is assumed: a job only
// waits for the previous round of its own instance, whose jobs all carry
// smaller numbers and were taken by CTAs that are already running.
//
// A job (date n, tile t) of instance i:
//   1. applies the exercise rule of date n+1 (coefficients published by the
//      previous round) to the tile's cash flows, or initialises them with the
//      payoff at maturity: in-the-money paths compacted per warp, each
//      decision first taken by a float screen with an error bound
//      (exercise.cuh); the items it leaves (exercise, or undecided) are
//      collected over the job and settled in the working precision a warp's
//      width at a time;
//   2. in a second pass over the tile, accumulates, over in-the-money paths
//      (compacted again), the 15
//      distinct monomials x^a w^b (a + b <= 4) that make up X^T X and the six
//      entries of X^T Y (register sums, a fixed-order sum over the lanes and
//      then over the warps: no atomics, so results do not depend on
//      scheduling);
//   3. writes the tile partial and arrives on the instance's counter.  The CTA
//      that arrives last sums the tile partials in tile order, solves the
//      normal equations by Cholesky in FP64 and publishes the coefficients.
// Every wait is bounded in time; on expiry the kernel records an error code
// and returns.
#include <atomic>
#include <cstdio>
#include <type_traits>

#include "checked.cuh"
#include "device_common.cuh"
#include "dfloat.cuh"
#include "exercise.cuh"
#include "kernels.h"
#include "plan.h"
#include "store16.cuh"

namespace lsmc {

namespace {

// monomial slot of x^a w^b
__host__ __device__ constexpr int mono(int a, int b) {
  return b == 0 ? a : b == 1 ? 5 + a : b == 2 ? 9 + a : b == 3 ? 12 + a : 14;
}

// Solve the B x B normal equations assembled from the monomial sums M and
// right-hand sides R.  Returns false (no exercise on this date) when fewer
// in-the-money paths than basis functions were seen, or when a Cholesky pivot
// is not above 1e-13 times the largest diagonal entry.
template <bool kNoDivide>
__device__ bool solve_normal_equations(int B, const double* M, const double* R,
                                       double beta[6]) {
  const int pa[6] = {0, 1, 2, 0, 1, 0};
  const int pb[6] = {0, 0, 0, 1, 1, 2};
  if (M[0] < (double)B) return false;
  double A[6][6], L[6][6];
  double maxdiag = 0.0;
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < B; ++j) A[i][j] = M[mono(pa[i] + pa[j], pb[i] + pb[j])];
  for (int i = 0; i < B; ++i) maxdiag = fmax(maxdiag, A[i][i]);
  // kNoDivide (the double-precision kernel): the solve is the critical path
  // of its regression's chain of dates and runs on one thread while the other
  // CTAs keep the FP64 pipe busy, where each dependent operation waits some
  // 200 cycles; one reciprocal square root per pivot gives both
  // L_jj = d / sqrt(d) and 1 / L_jj, and the substitutions multiply by the
  // reciprocals, so no division remains on the chain (within a few ulps of
  // the divided form): the last CTA's reduction and solve 33 -> 21 us, the
  // FP64 backward 1.4% faster.  The float-pair kernel, whose FP64 pipe is
  // idle, keeps the square root and the divisions (it measured 1.3% slower
  // with the reciprocals).
  double rinv[6];
  for (int j = 0; j < B; ++j) {
    double d = A[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 1e-13 * maxdiag)) return false;
    const double rj = kNoDivide ? rsqrt(d) : 0.0;
    L[j][j] = kNoDivide ? d * rj : sqrt(d);
    const double inv = kNoDivide ? rj : 1.0 / L[j][j];
    rinv[j] = inv;
    for (int i = j + 1; i < B; ++i) {
      double s = A[i][j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      L[i][j] = s * inv;
    }
  }
  double z[6];
  for (int i = 0; i < B; ++i) {
    double s = R[i];
    for (int k = 0; k < i; ++k) s -= L[i][k] * z[k];
    z[i] = kNoDivide ? s * rinv[i] : s / L[i][i];
  }
  for (int i = B - 1; i >= 0; --i) {
    double s = z[i];
    for (int k = i + 1; k < B; ++k) s -= L[k][i] * beta[k];
    beta[i] = kNoDivide ? s * rinv[i] : s / L[i][i];
  }
  for (int i = B; i < 6; ++i) beta[i] = 0.0;
  return true;
}

struct JobInfo {
  unsigned long long job;
  uint32_t inst, tile, round;
  int32_t abort;
};

}  // namespace

// Threads per CTA of the backward pass and resident CTAs per SM: 64 x 8 for
// double (shorter barriers around the FP64 pipe's work: the FP64 backward of
// the paper-size book 62.3 ms with 256 x 2, 59.4 with 128 x 4, 58.1 with
// 64 x 8), 256 x 2 for float pairs and float (which lose with 128).
// backward_block() on the host gives the same.
template <typename Real> struct BwdShape {
  static constexpr int kThreads = std::is_same<Real, double>::value ? 64 : kBlock;
  static constexpr int kMinBlocks = std::is_same<Real, double>::value ? 8 : 2;
};

// Derived per-instance constants: reciprocals of the basis scales, the
// exercise value at t_0, the S multiplier of every date (scale0 exp(n dr dt))
// and the discount factor of every date back to t_0 (exp(-r n dt)).
__global__ void setup_kernel(BwdInstance* inst, uint32_t n_inst CHK_PARAM) {
  const uint32_t i = blockIdx.x;
  if (i >= n_inst || !CHK_OK(chk, &inst[i], sizeof(BwdInstance))) return;
  BwdInstance& I = inst[i];
  if (threadIdx.x == 0) {
    I.disc = exp(-I.r * I.dt);
    I.disc_T = exp(-I.r * I.T);
    I.invK = 1.0 / I.K;
    I.inv_theta = 1.0 / I.theta;
    I.h0 = payoff_d(I.type, I.K, I.spot);
  }
  for (uint32_t n = threadIdx.x; n <= I.N; n += blockDim.x) {
    CHK_ST(chk, &I.scale_tab[n], I.dr_dt == 0.0 ? I.scale0 : I.scale0 * exp((double)n * I.dr_dt));
    CHK_ST(chk, &I.scale_tab[I.N + 1 + n], exp(-I.r * ((double)n * I.dt)));
  }
}

namespace {

// Knuth's two-sum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Sum of unevaluated float pairs (hi + lo): two-sum of the high parts, the
// low parts added to the error, renormalised.  About 44 bits survive.
__device__ __forceinline__ float2 pair_add(float2 x, float2 y) {
  float s, e;
  two_sum(x.x, y.x, s, e);
  e = __fadd_rn(e, __fadd_rn(x.y, y.y));
  const float hi = __fadd_rn(s, e);
  return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}


}  // namespace

namespace {

// Per-thread moment sums across the sub-tiles of a job.  Double precision
// adds into one double per sum.  Single precision sums at most 4 PPT paths in
// float, then folds that partial into an unevaluated pair (hi + lo) with
// Knuth's two-sum, so a job of many sub-tiles keeps about 44 bits beyond the
// partials' own rounding.
template <typename Real, int NA> struct Acc;
template <int NA> struct Acc<double, NA> {
  double s[NA];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NA; ++i) s[i] = 0.0;
  }
  __device__ __forceinline__ double* target() { return s; }
  __device__ __forceinline__ void fold() {}
};
template <int NA> struct Acc<df, NA> {
  df s[NA];  // float-pair accumulation needs no folding
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NA; ++i) s[i] = df(0.0f, 0.0f);
  }
  __device__ __forceinline__ df* target() { return s; }
  __device__ __forceinline__ void fold() {}
  __device__ __forceinline__ float2 pair(int i) const {
    const df t = quick_two_sum(s[i].hi, s[i].lo);
    return make_float2(t.hi, t.lo);
  }
};
template <int NA> struct Acc<float, NA> {
  float hi[NA], lo[NA], t[NA];
  __device__ __forceinline__ float2 pair(int i) const { return make_float2(hi[i], lo[i]); }
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NA; ++i) hi[i] = lo[i] = t[i] = 0.0f;
  }
  __device__ __forceinline__ float* target() { return t; }
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      float sum, err;
      two_sum(hi[i], t[i], sum, err);
      hi[i] = sum;
      lo[i] = __fadd_rn(lo[i], err);
      t[i] = 0.0f;
    }
  }
};

// Reduce-scatter of C per-lane doubles over the warp by recursive halving
// over the lane bits O, O / 2, ..., 1: at each level lane l and its partner
// l ^ O split the sums they still hold, the lane with the bit clear keeps the
// lower half and its partner the upper half (padded with zeros), and each
// adds the partner's copy of the half it keeps.  After the last level a lane
// holds one complete sum over the 32 lanes, summed in a fixed order; `idx` is
// its index (base + position), or -1 for a lane left with padding only.
template <int C, int O>
__device__ __forceinline__ void halving_sum(const double (&v)[C], int lane, int base, int real,
                                            double& out, int& idx) {
  constexpr int H = (C + 1) / 2;
  const bool upper = (lane & O) != 0;
  double nxt[H];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const double lo = v[i];
    const double hi = (H + i < C) ? v[(H + i < C) ? H + i : i] : 0.0;
    const double got = __shfl_xor_sync(0xffffffffu, upper ? lo : hi, O);
    nxt[i] = (upper ? hi : lo) + got;
  }
  const int nbase = upper ? base + H : base;
  const int nreal = upper ? (real > H ? real - H : 0) : (real < H ? real : H);
  if constexpr (O == 1) {
    static_assert(H == 1, "at most 32 sums");
    out = nxt[0];
    idx = nreal >= 1 ? nbase : -1;
  } else {
    halving_sum<H, O / 2>(nxt, lane, nbase, nreal, out, idx);
  }
}

}  // namespace

// Adds one in-the-money path to the per-thread moment sums: the 15
// monomials x^a w^b (a + b <= 4) of the centred basis variables
// x = S/K - 1, w = v/theta - 1 and the six products with the cash flow y.
// Every monomial of degree 3 or 4 is the product of two basis functions
// (x^3 = x^2 x, x^3 w = x^2 (x w), ...), so it is added as one fused
// multiply-add; the path count (monomial 1) is an integer.
template <typename Real, int BASIS, int NM>
__device__ __forceinline__ void accumulate_moments(Real* t, uint32_t& cnt, Real S, Real v, Real yv,
                                                   Real invK, Real invTh) {
  if constexpr (std::is_same<Real, float>::value) {
    // single precision (uncompacted, predicated loop): the count as a float
    // sum and the monomials as separate products schedule better there
    const Real x = qfma(S, invK, (Real)-1);
    const Real x2 = qmul(x, x), x3 = qmul(x2, x), x4 = qmul(x2, x2);
    qacc(t[0], (Real)1);
    qacc(t[1], x);
    qacc(t[2], x2);
    qacc(t[3], x3);
    qacc(t[4], x4);
    if (BASIS == kBasisSV2) {
      const Real w = qfma(v, invTh, (Real)-1);
      const Real w2 = qmul(w, w), w3 = qmul(w2, w), w4 = qmul(w2, w2);
      const Real xw = qmul(x, w);
      qacc(t[mono(0, 1)], w);
      qacc(t[mono(1, 1)], xw);
      qacc(t[mono(2, 1)], qmul(x2, w));
      qacc(t[mono(3, 1)], qmul(x3, w));
      qacc(t[mono(0, 2)], w2);
      qacc(t[mono(1, 2)], qmul(x, w2));
      qacc(t[mono(2, 2)], qmul(x2, w2));
      qacc(t[mono(0, 3)], w3);
      qacc(t[mono(1, 3)], qmul(x, w3));
      qacc(t[mono(0, 4)], w4);
      qacc(t[NM + 0], yv);
      qacc(t[NM + 1], qmul(x, yv));
      qacc(t[NM + 2], qmul(x2, yv));
      qacc(t[NM + 3], qmul(w, yv));
      qacc(t[NM + 4], qmul(xw, yv));
      qacc(t[NM + 5], qmul(w2, yv));
    } else {
      qacc(t[NM + 0], yv);
      qacc(t[NM + 1], qmul(x, yv));
      qacc(t[NM + 2], qmul(x2, yv));
    }
    return;
  }
  ++cnt;
  const Real x = qfma(S, invK, (Real)-1);
  const Real x2 = qmul(x, x);
  qacc(t[1], x);
  qacc(t[2], x2);
  qacc(t[3], qmul(x2, x));
  qacc(t[4], qmul(x2, x2));
  if (BASIS == kBasisSV2) {
    const Real w = qfma(v, invTh, (Real)-1);
    const Real w2 = qmul(w, w);
    const Real xw = qmul(x, w);
    qacc(t[mono(0, 1)], w);
    qacc(t[mono(1, 1)], xw);
    qacc(t[mono(2, 1)], qmul(x2, w));
    qacc(t[mono(3, 1)], qmul(x2, xw));
    qacc(t[mono(0, 2)], w2);
    qacc(t[mono(1, 2)], qmul(xw, w));
    qacc(t[mono(2, 2)], qmul(x2, w2));
    qacc(t[mono(0, 3)], qmul(w2, w));
    qacc(t[mono(1, 3)], qmul(xw, w2));
    qacc(t[mono(0, 4)], qmul(w2, w2));
    qacc(t[NM + 0], yv);
    qacc(t[NM + 1], qmul(x, yv));
    qacc(t[NM + 2], qmul(x2, yv));
    qacc(t[NM + 3], qmul(w, yv));
    qacc(t[NM + 4], qmul(xw, yv));
    qacc(t[NM + 5], qmul(w2, yv));
  } else {
    qacc(t[NM + 0], yv);
    qacc(t[NM + 1], qmul(x, yv));
    qacc(t[NM + 2], qmul(x2, yv));
  }
}

// Price and Greeks of one (request, strike) by central differences of its
// revaluation prices (the bump layout of the request's scenario table).
// Every operation rounds once (no contraction), so the Greeks kernel and the
// backward pass's per-request completion form the same bits.  kCg: the
// results were stored by other CTAs of the running launch (loads from L2).
template <bool kCg>
__device__ __forceinline__ bool form_greeks(const GreekOut& G, const BwdResult* res,
                                            DevResult& o CHK_PARAM) {
  for (int k = 0; k < kScCount; ++k)
    if (G.res[k] >= 0 && !CHK_OK(chk, &res[G.res[k]], sizeof(BwdResult))) return false;
  auto ld = [](const double* p) { return kCg ? __ldcg(p) : *p; };
  auto V = [&](int kind) { return ld(&res[G.res[kind]].price); };
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  const BwdResult* base = &res[G.res[kScBase]];
  o.price = ld(&base->price);
  o.price_se = ld(&base->se);
  o.european_price = ld(&base->euro);
  o.delta = o.gamma = o.vega = o.rho = o.theta = nan;
  // (V+ - V-) / (2 h): the central difference
  auto central = [&](int up, int dn, double h2) { return __ddiv_rn(__dsub_rn(V(up), V(dn)), h2); };
  if ((G.mask & 1u) && G.res[kScSUp] >= 0)
    o.delta = central(kScSUp, kScSDn, __dmul_rn(__dmul_rn(2.0, G.hS), G.S0));
  if (G.mask & 2u) {
    // (V+ - 2 V + V-) / h^2
    const bool own = G.res[kScSgUp] >= 0;
    if (own || G.res[kScSUp] >= 0) {
      const int up = own ? kScSgUp : kScSUp, dn = own ? kScSgDn : kScSDn;
      const double h = __dmul_rn(own ? G.hG : G.hS, G.S0);
      o.gamma = __ddiv_rn(__dadd_rn(__dsub_rn(V(up), __dmul_rn(2.0, V(kScBase))), V(dn)),
                          __dmul_rn(h, h));
    }
  }
  if ((G.mask & 4u) && G.res[kScVUp] >= 0)
    o.vega = central(kScVUp, kScVDn, __dmul_rn(__dmul_rn(2.0, G.hV), G.v0));
  if ((G.mask & 8u) && G.res[kScRUp] >= 0) o.rho = central(kScRUp, kScRDn, __dmul_rn(2.0, G.dR));
  if ((G.mask & 16u) && G.res[kScTDn] >= 0)
    o.theta = central(kScTDn, kScTUp, __dmul_rn(2.0, G.dT));
  uint32_t sing = 0, nrev = 0;
  double ties = 0.0;
  for (int k = 0; k < kScCount; ++k)
    if (G.res[k] >= 0) {
      const BwdResult* r = &res[G.res[k]];
      sing += kCg ? __ldcg(&r->singular) : r->singular;
      ties = __dadd_rn(ties, ld(&r->ties));
      ++nrev;
    }
  o.n_singular_solves = sing;
  o.n_revaluations = nrev;
  o.status = sing ? 1 : 0;
  o.n_near_ties = (uint32_t)ties;
  return true;
}

// Per-request completion (serving), by thread 0 of a CTA that has stored the
// final result of one of request q's instances: the request's last instance
// to finish forms its prices and Greeks, writes them to the host-mapped
// array and then raises the request's host-mapped flag.  The results of the
// other instances were stored before their CTAs' fenced arrivals on the
// counter, so the last arrival reads them all.
__device__ __forceinline__ void finish_request(const BwdArgs& a, uint32_t q) {
  const uint32_t* info = a.req_info + 3 * (size_t)q;
  if (!CHK_OK(a.chk, info, 3 * sizeof(uint32_t)) ||
      !CHK_OK(a.chk, &a.req_count[q], sizeof(uint32_t)) ||
      !CHK_OK(a.chk, &a.flag_host[q], sizeof(uint32_t)))
    return;
  __threadfence();
  if (atomicAdd(&a.req_count[q], 1u) + 1u != info[0]) return;
  __threadfence();
  for (uint32_t g = info[1]; g < info[1] + info[2]; ++g) {
    DevResult o;
    if (!CHK_OK(a.chk, &a.greeks[g], sizeof(GreekOut)) ||
        !form_greeks<true>(a.greeks[g], a.results, o CHK_ARG(a.chk)))
      return;
    CHK_ST(a.chk, &a.out_host[g], o);
  }
  __threadfence_system();
  *(volatile uint32_t*)&a.flag_host[q] = 1u;
}

// Per-warp buffers of the backward kernel (dynamic shared memory): the row
// values (e or S, and v) of the in-the-money paths compacted for the
// exercise test and their origins (k * 32 + lane); the row values and cash
// flows of those compacted for the moment sums (room for a sub-tile plus the
// fewer than 32 items carried from the previous one; the float-pair job-end
// reduction reuses this space); the exercise items the float screen did not
// settle, collected over a job (the same room): row values, and the path's
// offset in the job tile | the screen's verdict << 30.
template <typename Real, int PPT>
struct BwdWarpBufs {
  static constexpr int kCap = 32 * PPT;
  Real xs[kCap];
  Real xv[kCap];
  Real m[3][kCap + 32];
  unsigned short co[kCap];
  Real xe[kCap + 32];
  Real xw[kCap + 32];
  uint32_t xo[kCap + 32];
};

// Compaction buffer items.  With a 16-bit store in double precision the row
// values stay floats (exact: every 16-bit value is a float) until the dense
// loops, so the float -> double conversions, which run on the FP64 pipe,
// happen once per in-the-money item rather than once per path; such an item
// sits in the low half of its double slot.
template <typename Real, typename LoadT>
__device__ __forceinline__ void put_item(Real* buf, int i, LoadT x) {
  if constexpr (std::is_same<Real, LoadT>::value) buf[i] = x;
  else reinterpret_cast<float*>(buf + i)[0] = x;
}
template <typename Real, typename LoadT>
__device__ __forceinline__ Real get_item(const Real* buf, int i) {
  if constexpr (std::is_same<Real, LoadT>::value) return buf[i];
  else return (Real)reinterpret_cast<const float*>(buf + i)[0];
}
template <typename Real, typename LoadT>
__device__ __forceinline__ float item_float(const Real* buf, int i) {
  if constexpr (std::is_same<Real, LoadT>::value) return approx_float(buf[i]);
  else return reinterpret_cast<const float*>(buf + i)[0];
}

// Cash flows are kept discounted to t_0: Z = h(S_tau) exp(-r tau dt) for the
// current exercise time tau.  The regression target of date n, the cash flow
// discounted to t_n, is Z exp(r n dt): the same factor for every path, so the
// regression runs on Z and the exercise test compares h exp(-r n dt) with the
// fitted value in the same units.  Z changes only where a path exercises.
//
// A job covers `I.sub` sub-tiles of kBT * PPT paths (kBT threads per CTA:
// BwdShape): the wait for the
// previous round, the block reduction and the arrival are paid once per job.
template <typename Real, int BASIS, int PPT, int FMT>
__global__ void __launch_bounds__(BwdShape<Real>::kThreads, BwdShape<Real>::kMinBlocks)
backward_kernel(BwdArgs a) {
  constexpr int kBT = BwdShape<Real>::kThreads;
  using RR = RowRead<Real, FMT>;  // the E/V rows' elements and their widening
  using St = typename RR::raw;
  // double with a 16-bit store: row values kept as floats until the dense loops
  constexpr bool kNarrow64 = std::is_same<Real, double>::value && FMT != kStoreNative;
  using LoadT = typename std::conditional<kNarrow64, float, Real>::type;
  using RF = RowRead<LoadT, FMT>;
  constexpr int NB = BASIS == kBasisSV2 ? 6 : 3;      // basis functions
  constexpr int NM = BASIS == kBasisSV2 ? 15 : 5;     // distinct monomials
  constexpr int NA = NM + NB;                         // register sums
  constexpr int TILE0 = kBT * PPT;
  constexpr int NW = kBT / 32;

  __shared__ JobInfo s_job;
  __shared__ double s_beta[6];
  __shared__ int s_beta_ok;
  __shared__ int s_last;
  __shared__ double s_red[NW][kNSum];
  __shared__ float2 s_redf[NW][NA];   // single precision: per-warp pair sums
  __shared__ double s_chunk[NW][kNSum];
  __shared__ double s_sum[kNSum];
  __shared__ Real s_c[16];            // per-job constants, converted once
  __shared__ long long s_thr[2];      // double: in-the-money thresholds of dates n + 1, n
  __shared__ int s_thrf[2];           // the same for float row values (16-bit store)
  __shared__ df s_thrdf[2];           // float pairs: the thresholds K / s of dates n + 1, n
  __shared__ ScreenConsts s_q;        // the exercise test of date n + 1 in float
  // per-warp compaction of in-the-money paths (dynamic shared memory, one
  // BwdWarpBufs per warp): the heavy arithmetic runs on dense lists instead
  // of on lanes that are mostly out of the money
  using Bufs = BwdWarpBufs<Real, PPT>;
  extern __shared__ __align__(16) unsigned char bwd_dyn[];
  Bufs& wb = reinterpret_cast<Bufs*>(bwd_dyn)[threadIdx.x >> 5];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // single precision and float pairs reduce through float pairs; double
  // precision through doubles
  constexpr bool kSingle = !std::is_same<Real, double>::value;
  // compaction pays where the in-the-money arithmetic is heavy (double and
  // float pairs); plain floats are bound by loads and stay uncompacted
  constexpr bool kCompact = !std::is_same<Real, float>::value;
  // double and float pairs: the in-the-money test needs no product (a
  // threshold on the stored value), so the compaction buffers hold the
  // stored value and S = s e is formed on the dense lists, where no lane idles
  constexpr bool kProdLate = kCompact;
  // Job taking and decoding by thread 0, when the CTA has arrived with its
  // previous job: a job is taken only once the CTA can start it.
  auto decode = [&]() {
    JobInfo ji;
    ji.abort = 0;
    ji.round = ji.inst = ji.tile = 0;
    ji.job = ld_volatile(&a.ctl->error) != 0 ? a.total_jobs
                                             : atomicAdd(&a.ctl->next_job, 1ull);
    if (ji.job >= a.total_jobs) {
      ji.abort = 1;
    } else {
      // round: last r with round_off[r] <= job
      uint32_t lo = 0, hi = a.n_rounds;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        if (CHK_LD(a.chk, &a.round_off[mid]) <= ji.job) lo = mid; else hi = mid;
      }
      const uint32_t local = (uint32_t)(ji.job - CHK_LD(a.chk, &a.round_off[lo]));
      uint32_t klo = 0, khi = CHK_LD(a.chk, &a.active[lo]);
      while (khi - klo > 1) {
        const uint32_t mid = (klo + khi) / 2;
        if (CHK_LD(a.chk, &a.cum_tiles[mid]) <= local) klo = mid; else khi = mid;
      }
      ji.round = lo;
      ji.inst = klo;
      ji.tile = local - CHK_LD(a.chk, &a.cum_tiles[klo]);
      // the job's instance and state must lie in the tables
      if (!CHK_OK(a.chk, &a.inst[klo], sizeof(BwdInstance)) ||
          !CHK_OK(a.chk, &a.state[klo], sizeof(BwdState)))
        ji.abort = 1;
    }
    s_job = ji;
  };
  // the control word (job counter, error word) must lie in the plan
  if (!CHK_OK(a.chk, a.ctl, sizeof(Control))) return;
  if (tid == 0) decode();
  __syncthreads();

  for (;;) {
    const JobInfo ji = s_job;
    if (ji.abort) return;

    const BwdInstance& I = a.inst[ji.inst];
    BwdState* st = &a.state[ji.inst];
    const uint32_t N = I.N, P = I.P, r = ji.round;
    const size_t ld = I.ld;
    const St* E = (const St*)I.E;
    const St* V = (const St*)I.V;
    Real* Z = (Real*)I.Y;
    const double* stab = I.scale_tab;          // S multipliers, dates 0..N
    const double* dtab = I.scale_tab + N + 1;  // discount to t_0, dates 0..N
    const int type = I.type;
    const bool european = I.style == kEuropean;
    const bool final_job = european || r == N - 1;
    // regression date of this round (0 for the estimator round)
    const uint32_t n = european ? 0 : N - 1 - r;
    const bool first = european || r == 0;  // cash flows start at the maturity payoff
    const uint32_t sub = I.sub;
    const uint32_t tile_base = ji.tile * (sub * TILE0);

    // ---- warp 0: wait for the exercise rule of date n + 1, then convert the
    // per-job constants to the working precision once ------------------------
    if (warp == 0) {
      if (tid == 0) {
        int ok = 1;
        if (!first) {
          const unsigned long long t0 = global_timer_ns();
          unsigned spins = 0, ns = 32;
          while (ld_acquire_gpu(&st->ready) < r) {
            // back off (32 ns doubling to 512 ns); the error word and the
            // clock are read every 32nd time
            __nanosleep(ns);
            ns = ns < 512 ? 2 * ns : 512;
            if ((++spins & 31) == 0) {
              if (ld_volatile(&a.ctl->error) != 0) { ok = 0; break; }
              if (spins > (1u << 26) || global_timer_ns() - t0 > a.timeout_ns) {
                atomicCAS(&a.ctl->error, 0u, (uint32_t)kDevErrTimeout);
                a.ctl->error_info = ji.inst;
                ok = 0;
                break;
              }
            }
          }
          if (ok) {
            __threadfence();
            s_beta_ok = (int)__ldcg(&st->beta_ok);
            for (int i = 0; i < 6; ++i) s_beta[i] = __ldcg(&st->beta[i]);
          }
        }
        s_last = ok ? 0 : -1;
      }
      __syncwarp();
      if (lane < 16) {
        double v;
        switch (lane) {
          case 6: v = CHK_LD(a.chk, &stab[n + 1]); break;
          case 7: v = CHK_LD(a.chk, &dtab[n + 1]); break;
          case 8: v = CHK_LD(a.chk, &stab[N]); break;
          case 9: v = CHK_LD(a.chk, &stab[n]); break;
          case 10: v = I.K; break;
          case 11: v = I.invK; break;
          case 12: v = I.inv_theta; break;
          // discount factors as unevaluated pairs (hi + lo): a cash flow is
          // h * hi + h * lo, one rounding, with no bias shared by the paths
          // that exercise on the same date
          case 13: {
            const double d = CHK_LD(a.chk, &dtab[n + 1]);
            v = d - (double)(Real)d;
            break;
          }
          case 14: v = CHK_LD(a.chk, &dtab[N]); break;
          case 15: {
            const double d = CHK_LD(a.chk, &dtab[N]);
            v = d - (double)(Real)d;
            break;
          }
          default: v = first ? 0.0 : s_beta[lane]; break;
        }
        s_c[lane] = (Real)v;
      } else if (kProdLate && lane < 18) {
        const double sv = CHK_LD(a.chk, lane == 16 ? &stab[n + 1] : &stab[n]);
        if constexpr (std::is_same<Real, double>::value) {
          const double T = itm_threshold(type, sv, I.K);
          s_thr[lane - 16] = __double_as_longlong(T);
          // float e: e < T iff e < (T rounded up to a float); e > T iff e > (T rounded down)
          if constexpr (kNarrow64)
            s_thrf[lane - 16] =
                __float_as_int(type == kPut ? __double2float_ru(T) : __double2float_rd(T));
        } else {
          // float pairs: S = s e < K where e < K / s (put), > for a call; the
          // two tests can differ only where s e lies within the pairs'
          // rounding (about 1e-14 relative) of K
          s_thrdf[lane - 16] = df(I.K / sv);
        }
      }
      __syncwarp();
      // the compaction buffers hold the row value e (double) or S itself
      if (kCompact && lane == 0)
        make_screen<BASIS, Real>(s_q, s_c, kProdLate ? s_c[6] : (Real)1, s_c[10], s_c[11],
                                 s_c[12], s_c[7]);
    }
    __syncthreads();
    if (s_last < 0) return;
    const int bok = first ? 0 : s_beta_ok;
    Real b[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) b[i] = s_c[i];
    const Real s1 = s_c[6], d1 = s_c[7], sN = s_c[8], s0 = s_c[9];
    const Real K = s_c[10], invK = s_c[11], invTh = s_c[12];
    const Real d1lo = s_c[13], dNhi = s_c[14], dNlo = s_c[15];
    // double: S = RN(s e) is in the money exactly when e's bits pass the
    // date's threshold, so only in-the-money paths pay for the product
    const long long thr1 = std::is_same<Real, double>::value ? s_thr[0] : 0;
    const long long thr0 = std::is_same<Real, double>::value ? s_thr[1] : 0;
    // the moment items hold e (double) or S: x = e (s0 / K) - 1 or S / K - 1
    const Real xK0 = kProdLate ? s0 * invK : invK;
    // row of date d at index d - a.row0 (rows of dates 1..N, or one segment)
    const ptrdiff_t r0 = (ptrdiff_t)a.row0;
    const St* EN = E + ((ptrdiff_t)N - r0) * (ptrdiff_t)ld;
    const St* E1 = E + ((ptrdiff_t)n + 1 - r0) * (ptrdiff_t)ld;                    // date n + 1
    const St* V1 = BASIS == kBasisSV2 ? V + ((ptrdiff_t)n + 1 - r0) * (ptrdiff_t)ld : nullptr;
    const St* E0 = final_job ? nullptr : E + ((ptrdiff_t)n - r0) * (ptrdiff_t)ld;  // date n
    const St* V0 = (BASIS == kBasisSV2 && !final_job)
                         ? V + ((ptrdiff_t)n - r0) * (ptrdiff_t)ld : nullptr;

    Acc<Real, NA> acc;
    acc.zero();
    uint32_t n_itm = 0;  // in-the-money paths of this thread (monomial 1)
    double euro = 0.0, sy = 0.0, sy2 = 0.0;
    uint32_t ties = 0;

    const unsigned lane_lt = (1u << lane) - 1u;
    if constexpr (!kCompact) {
      // single precision: one predicated pass per sub-tile (bound by loads)
      for (uint32_t sb = 0; sb < sub; ++sb) {
        const uint32_t sub_base = tile_base + sb * TILE0;
        if (sub_base >= P) break;  // uniform across the CTA
        const uint32_t p_base = sub_base + tid;
        // every load of the sub-tile is issued before any arithmetic, so each
        // thread has up to 5 * PPT independent loads in flight
        Real zr[PPT];
        St e1r[PPT], v1r[PPT], e0r[PPT], v0r[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          const uint32_t p = p_base + k * kBT;
          zr[k] = (Real)0;
          e1r[k] = v1r[k] = e0r[k] = v0r[k] = (St)0;
          if (p < P) {
            if (first) {
              e1r[k] = CHK_LD(a.chk, &EN[p]);
            } else {
              zr[k] = CHK_OK(a.chk, Z + p, sizeof(Real)) ? ld_cg(Z + p) : (Real)0;
              if (bok) {
                e1r[k] = CHK_LD(a.chk, &E1[p]);
                if (BASIS == kBasisSV2) v1r[k] = CHK_LD(a.chk, &V1[p]);
              }
            }
            if (!final_job) {
              e0r[k] = CHK_LD(a.chk, &E0[p]);
              if (BASIS == kBasisSV2) v0r[k] = CHK_LD(a.chk, &V0[p]);
            }
          }
        }
        LoadT e1[PPT], v1[PPT], e0[PPT], v0[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          e1[k] = RF::widen(e1r[k]);
          v1[k] = RF::widen(v1r[k]);
          e0[k] = RF::widen(e0r[k]);
          v0[k] = RF::widen(v0r[k]);
        }
        Real z[PPT];
        if (first) {
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            const uint32_t p = p_base + k * kBT;
            z[k] = (Real)0;
            if (p < P) {
              const Real h = payoff<Real>(type, K, sN * (Real)e1[k]);
              z[k] = fma(h, dNhi, h * dNlo);
              euro += (double)z[k];
              if (!final_job) CHK_ST(a.chk, &Z[p], z[k]);
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < PPT; ++k) z[k] = zr[k];
          if (bok) {
            // exercise at date n + 1 where the discounted payoff beats the
            // fitted continuation value (basis centred at the strike and theta)
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
              const uint32_t p = p_base + k * kBT;
              const Real S = s1 * e1[k];
              if (p < P && in_money<Real>(type, K, S)) {
                const Real h = intrinsic<Real>(type, K, S);
                const Real x = qfma(S, invK, (Real)-1);
                Real c = qfma(qfma(b[2], x, b[1]), x, b[0]);
                if (BASIS == kBasisSV2) {
                  const Real w = qfma((Real)v1[k], invTh, (Real)-1);
                  c = qfma(qfma(b[5], w, qfma(b[4], x, b[3])), w, c);
                }
                const Real hd = qmul(h, d1);
                bool exercise, tie;
                decide<Real>(hd, c, exercise, tie);
                if (tie) ++ties;
                if (exercise) {
                  const Real hz = fma(h, d1, h * d1lo);
                  z[k] = hz;
                  if (!final_job) CHK_ST(a.chk, &Z[p], hz);
                }
              }
            }
          }
        }
        if (final_job) {
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            const uint32_t p = p_base + k * kBT;
            if (p < P) {
              const double zv = (double)z[k];
              sy += zv;
              sy2 += zv * zv;
            }
          }
        } else {
          // moment sums of date n over the in-the-money paths
          Real* t = acc.target();
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            const uint32_t p = p_base + k * kBT;
            const Real S = s0 * e0[k];
            if (p < P && in_money<Real>(type, K, S)) {
              accumulate_moments<Real, BASIS, NM>(t, n_itm, S, v0[k], z[k], invK, invTh);
            }
          }
          // the float partial sums cover four sub-tiles (4 PPT paths a lane)
          // before they are folded into the pairs: at 1,048,576 paths the
          // single-precision backward 83.5 ms with a fold per sub-tile, 79.8
          // with one per two, 77.9 with one per four
          if ((sb & 3u) == 3u) acc.fold();
        }
      }
      acc.fold();
    } else {
      // ---- pass 1: the exercise rule of date n + 1 (or the payoff at
      // maturity) on every sub-tile.  In-the-money paths are compacted per
      // warp and screened in float; the items the screen does not settle as
      // continuing (exercise, or undecided) are collected over the whole job
      // and settled in the working precision a warp's width at a time, the
      // remainder carried to the next sub-tile, so those lanes stay busy as
      // well (an FP64 warp instruction costs the same whatever its active
      // lanes).  The cash flows after the rule are in Z for pass 2.
      if (first || bok) {
        Real* cs = wb.xs;
        Real* cv = wb.xv;
        unsigned short* co = wb.co;
        // one collected item: its row values (as the compaction buffers hold
        // them), its path's offset in the job tile and the screen's verdict
        auto settle = [&](int j) {
          const uint32_t code = wb.xo[j];
          const int pre = (int)(code >> 30);
          const uint32_t p = tile_base + (code & 0x3fffffffu);
          const Real S = kProdLate ? s1 * get_item<Real, LoadT>(wb.xe, j) : wb.xe[j];
          const Real h = intrinsic<Real>(type, K, S);
          const Real hd = qmul(h, d1);
          bool exercise = pre == 1;
          if (pre == 2) {
            const Real x = qfma(S, invK, (Real)-1);
            Real c = qfma(qfma(b[2], x, b[1]), x, b[0]);
            if (BASIS == kBasisSV2) {
              const Real w = qfma(get_item<Real, LoadT>(wb.xw, j), invTh, (Real)-1);
              c = qfma(qfma(b[5], w, qfma(b[4], x, b[3])), w, c);
            }
            bool tie;
            decide<Real>(hd, c, exercise, tie);
            if (tie) ++ties;
          }
          if (exercise) {
            Real hz;
            if constexpr (std::is_same<Real, df>::value) {
              hz = quick_two_sum(hd.hi, hd.lo);
            } else {
              hz = fma(h, d1, h * d1lo);
            }
            CHK_ST(a.chk, &Z[p], hz);
          }
        };
        int xn = 0;  // collected items not yet settled (fewer than 32)
        for (uint32_t sb = 0; sb < sub; ++sb) {
          const uint32_t sub_base = tile_base + sb * TILE0;
          if (sub_base >= P) break;  // uniform across the CTA
          const uint32_t p_base = sub_base + tid;
          St e1r[PPT], v1r[PPT];
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            const uint32_t p = p_base + k * kBT;
            e1r[k] = v1r[k] = (St)0;
            if (p < P) {
              if (first) {
                e1r[k] = CHK_LD(a.chk, &EN[p]);
              } else {
                e1r[k] = CHK_LD(a.chk, &E1[p]);
                if (BASIS == kBasisSV2) v1r[k] = CHK_LD(a.chk, &V1[p]);
              }
            }
          }
          LoadT e1[PPT], v1[PPT];
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            e1[k] = RF::widen(e1r[k]);
            v1[k] = RF::widen(v1r[k]);
          }
          if (first) {
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
              const uint32_t p = p_base + k * kBT;
              if (p < P) {
                const Real h = payoff<Real>(type, K, sN * (Real)e1[k]);
                const Real z = fma(h, dNhi, h * dNlo);
                euro += (double)z;
                CHK_ST(a.chk, &Z[p], z);
              }
            }
            continue;
          }
          int cnt = 0;
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            const uint32_t p = p_base + k * kBT;
            bool itm;
            if constexpr (kNarrow64) {
              const int eb = __float_as_int(e1[k]);
              itm = p < P && (type == kPut ? eb < s_thrf[0] : eb > s_thrf[0]);
            } else if constexpr (std::is_same<Real, df>::value) {
              itm = p < P && (type == kPut ? e1[k] < s_thrdf[0] : s_thrdf[0] < e1[k]);
            } else {
              itm = p < P && itm_test(type, K, s1, e1[k], thr1);
            }
            const unsigned m = __ballot_sync(0xffffffffu, itm);
            if (itm) {
              const int pos = cnt + __popc(m & lane_lt);
              if constexpr (kProdLate) put_item<Real, LoadT>(cs, pos, e1[k]);
              else cs[pos] = s1 * e1[k];
              if (BASIS == kBasisSV2) put_item<Real, LoadT>(cv, pos, v1[k]);
              co[pos] = (unsigned short)(k * 32 + lane);
            }
            cnt += __popc(m);
          }
          __syncwarp();
          for (int j0 = 0; j0 < cnt; j0 += 32) {
            const int j = j0 + lane;
            int pre = 0;
            if (j < cnt)
              pre = exercise_screen<BASIS>(s_q, type, item_float<Real, LoadT>(cs, j),
                                           BASIS == kBasisSV2 ? item_float<Real, LoadT>(cv, j)
                                                              : 0.0f);
            const unsigned m = __ballot_sync(0xffffffffu, pre != 0);
            if (pre != 0) {
              const int q = xn + __popc(m & lane_lt);
              const int o = co[j];
              wb.xe[q] = cs[j];
              if (BASIS == kBasisSV2) wb.xw[q] = cv[j];
              wb.xo[q] = (sb * TILE0 + (uint32_t)(o >> 5) * kBT + warp * 32 + (o & 31)) |
                         ((uint32_t)pre << 30);
            }
            xn += __popc(m);
          }
          __syncwarp();
          const int full = xn & ~31;
          for (int j = lane; j < full; j += 32) settle(j);
          const int rem = xn - full;
          Real t0 = (Real)0, t1 = (Real)0;
          uint32_t t2 = 0;
          if (lane < rem) {
            t0 = wb.xe[full + lane];
            if (BASIS == kBasisSV2) t1 = wb.xw[full + lane];
            t2 = wb.xo[full + lane];
          }
          __syncwarp();
          if (lane < rem) {
            wb.xe[lane] = t0;
            if (BASIS == kBasisSV2) wb.xw[lane] = t1;
            wb.xo[lane] = t2;
          }
          __syncwarp();
          xn = rem;
        }
        if (lane < xn) settle(lane);  // the items left from the last sub-tile
        // the cash flows stored above are read back by other lanes of the warp
        __threadfence_block();
        __syncwarp();
      }

      // ---- pass 2: the moment sums of date n over the in-the-money paths
      // (the estimator sums in the last round) with the cash flows after the
      // rule; only whole warps of compacted items are summed, the rest is
      // carried to the next sub-tile (or summed at the end of the job)
      Real* ms = wb.m[0];
      Real* mv = wb.m[1];
      Real* my = wb.m[2];
      int mcarry = 0;  // compacted moment items carried to the next sub-tile
      for (uint32_t sb = 0; sb < sub; ++sb) {
        const uint32_t sub_base = tile_base + sb * TILE0;
        if (sub_base >= P) break;  // uniform across the CTA
        const uint32_t p_base = sub_base + tid;
        Real z[PPT];
        St e0r[PPT], v0r[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          const uint32_t p = p_base + k * kBT;
          z[k] = (Real)0;
          e0r[k] = v0r[k] = (St)0;
          if (p < P) {
            z[k] = CHK_OK(a.chk, Z + p, sizeof(Real)) ? ld_cg(Z + p) : (Real)0;
            if (!final_job) {
              e0r[k] = CHK_LD(a.chk, &E0[p]);
              if (BASIS == kBasisSV2) v0r[k] = CHK_LD(a.chk, &V0[p]);
            }
          }
        }
        if (final_job) {
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            const uint32_t p = p_base + k * kBT;
            if (p < P) {
              const double zv = (double)z[k];
              sy += zv;
              sy2 += zv * zv;
            }
          }
          continue;
        }
        LoadT e0[PPT], v0[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          e0[k] = RF::widen(e0r[k]);
          v0[k] = RF::widen(v0r[k]);
        }
        int cnt = mcarry;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          const uint32_t p = p_base + k * kBT;
          bool itm;
          if constexpr (kNarrow64) {
            const int eb = __float_as_int(e0[k]);
            itm = p < P && (type == kPut ? eb < s_thrf[1] : eb > s_thrf[1]);
          } else if constexpr (std::is_same<Real, df>::value) {
            itm = p < P && (type == kPut ? e0[k] < s_thrdf[1] : s_thrdf[1] < e0[k]);
          } else {
            itm = p < P && itm_test(type, K, s0, e0[k], thr0);
          }
          const unsigned m = __ballot_sync(0xffffffffu, itm);
          if (itm) {
            const int pos = cnt + __popc(m & lane_lt);
            if constexpr (kProdLate) put_item<Real, LoadT>(ms, pos, e0[k]);
            else ms[pos] = s0 * e0[k];
            if (BASIS == kBasisSV2) put_item<Real, LoadT>(mv, pos, v0[k]);
            my[pos] = z[k];
          }
          cnt += __popc(m);
        }
        __syncwarp();
        Real* t = acc.target();
        const int full = cnt & ~31;
        for (int j = lane; j < full; j += 32)
          accumulate_moments<Real, BASIS, NM>(t, n_itm, get_item<Real, LoadT>(ms, j),
                                              get_item<Real, LoadT>(mv, j), my[j], xK0, invTh);
        mcarry = cnt - full;
        Real r0 = (Real)0, r1 = (Real)0, r2 = (Real)0;
        if (lane < mcarry) {
          r0 = ms[full + lane];
          if (BASIS == kBasisSV2) r1 = mv[full + lane];
          r2 = my[full + lane];
        }
        __syncwarp();
        if (lane < mcarry) {
          ms[lane] = r0;
          if (BASIS == kBasisSV2) mv[lane] = r1;
          my[lane] = r2;
        }
        __syncwarp();
        acc.fold();
      }
      if (mcarry > 0) {  // the carried moment items of the last sub-tile
        if (lane < mcarry)
          accumulate_moments<Real, BASIS, NM>(acc.target(), n_itm, get_item<Real, LoadT>(ms, lane),
                                              get_item<Real, LoadT>(mv, lane), my[lane], xK0,
                                              invTh);
        __syncwarp();
      }
    }

    // ---- block reduction into the tile partial --------------------------------
    // per warp first, in a fixed order: double precision by a reduce-scatter
    // over shuffles; the float-pair sums through shared memory transposed (a
    // row per sum, padded against bank conflicts, in the warp's compaction
    // buffers), lane i adding row i in lane order
    if (final_job) {
      sy = warp_sum(sy);
      sy2 = warp_sum(sy2);
    } else if constexpr (!kSingle) {
      // double: reduce-scatter by recursive halving, all lanes busy (an FP64
      // warp instruction takes the same pipe time whatever its active
      // lanes): about NA adds per lane in place of 31 per sum on NA lanes
      double vs[NA];
#pragma unroll
      for (int i = 0; i < NA; ++i) vs[i] = i == 0 ? (double)n_itm : acc.s[i];  // the count: an integer
      double out;
      int i;
      halving_sum<NA, 16>(vs, lane, 0, NA, out, i);
      if (i >= 0) s_red[warp][i < NM ? i : kSlotRhs + (i - NM)] = out;
    } else {
      // rows per pass: as many as the warp's moment buffers hold
      constexpr int RROWS = (int)(sizeof(wb.m) / (33 * sizeof(float2)));
      static_assert(RROWS >= 1 && RROWS <= 32, "reduction rows per pass");
      float2(*red)[33] = reinterpret_cast<float2(*)[33]>(&wb.m[0][0]);
      __syncwarp();
#pragma unroll
      for (int a0 = 0; a0 < NA; a0 += RROWS) {
#pragma unroll
        for (int i = a0; i < NA && i < a0 + RROWS; ++i) {
          // the path count: an integer, except in single precision
          if constexpr (std::is_same<Real, float>::value)
            red[i - a0][lane] = acc.pair(i);
          else
            red[i - a0][lane] = i == 0 ? make_float2((float)n_itm, 0.0f) : acc.pair(i);
        }
        __syncwarp();
        const int i = a0 + lane;
        if (lane < RROWS && i < NA) {
          float2 pr = red[lane][0];
          for (int l = 1; l < 32; ++l) pr = pair_add(pr, red[lane][l]);
          s_redf[warp][i] = pr;
        }
        __syncwarp();
      }
    }
    if (first) euro = warp_sum(euro);
    ties = __reduce_add_sync(0xffffffffu, ties);
    if (lane == 0) {
      s_red[warp][kSlotEuro] = euro;
      s_red[warp][kSlotTies] = (double)ties;
      s_red[warp][kSlotSumY] = sy;
      s_red[warp][kSlotSumY2] = sy2;
    }
    __syncthreads();
    if (tid < kNSum) {
      const bool moment = tid < NM || (tid >= kSlotRhs && tid < kSlotRhs + NB);
      const bool used = final_job ? tid >= kSlotEuro
                                  : (moment || tid == kSlotEuro || tid == kSlotTies);
      double v = 0.0;
      if (used) {
        if (kSingle && moment) {
          const int i = tid < NM ? tid : NM + (tid - kSlotRhs);
          float2 pr = make_float2(0.0f, 0.0f);
          for (int w = 0; w < NW; ++w) pr = pair_add(pr, s_redf[w][i]);
          v = (double)pr.x + (double)pr.y;
        } else {
          for (int w = 0; w < NW; ++w) v += s_red[w][tid];
        }
      }
      CHK_ST(a.chk, &I.partial[(size_t)ji.tile * kNSum + tid], v);
    }

    // ---- arrive; the last tile of this round reduces and solves ---------------
    // the partial was written by warp 0 alone and every other write of this
    // job is ordered before the reduction barrier above, so a warp-level
    // sync suffices before the fence and the arrival
    if (warp == 0) {
      __syncwarp();
      if (tid == 0) {
        __threadfence();
        const uint32_t old = atomicAdd(&st->arrive, 1u);
        s_last = (old + 1 == (r + 1) * I.tiles) ? 1 : 0;
        if (s_last) __threadfence();
        decode();
      }
    }
    __syncthreads();
    if (!s_last) continue;

    {
      // fixed-order sum of the tile partials: a contiguous chunk of tiles per
      // warp, a slot per lane, then the chunks in order
      const uint32_t tiles = I.tiles;
      const uint32_t per = (tiles + NW - 1) / NW;
      if (lane < kNSum) {
        double v = 0.0;
        const uint32_t t0 = warp * per, t1 = min(tiles, t0 + per);
        for (uint32_t t = t0; t < t1; ++t)
          if (CHK_OK(a.chk, &I.partial[(size_t)t * kNSum + lane], sizeof(double)))
            v += __ldcg(&I.partial[(size_t)t * kNSum + lane]);
        s_chunk[warp][lane] = v;
      }
      __syncthreads();
      if (tid < kNSum) {
        double v = 0.0;
        for (int w = 0; w < NW; ++w) v += s_chunk[w][tid];
        s_sum[tid] = v;
      }
      __syncthreads();
    }
    if (tid == 0) {
      if (final_job) {
        BwdResult res;
        const double Pd = (double)P;
        const double mean = s_sum[kSlotSumY] / Pd;
        const double var = P > 1 ? (s_sum[kSlotSumY2] - Pd * mean * mean) / (Pd - 1.0) : 0.0;
        const double euro_sum = first ? s_sum[kSlotEuro] : __ldcg(&st->euro_sum);
        res.cont = mean;
        res.se = var > 0.0 ? sqrt(var / Pd) : 0.0;
        res.euro = euro_sum / Pd;
        res.price = european ? mean : fmax(I.h0, mean);
        res.itm = __ldcg(&st->itm);
        res.ties = __ldcg(&st->ties) + s_sum[kSlotTies];
        res.singular = __ldcg(&st->singular);
        res.done = 1;
        CHK_ST(a.chk, &a.results[I.out_index], res);
        if (a.flag_host != nullptr) finish_request(a, I.req);
      } else {
        double beta[6];
        const bool ok = solve_normal_equations<std::is_same<Real, double>::value>(
            NB, s_sum, s_sum + kSlotRhs, beta);
        if (r == 0) st->euro_sum = s_sum[kSlotEuro];
        st->itm = __ldcg(&st->itm) + s_sum[0];
        st->ties = __ldcg(&st->ties) + s_sum[kSlotTies];
        if (!ok) st->singular = __ldcg(&st->singular) + 1u;
        st->beta_ok = ok ? 1u : 0u;
        for (int i = 0; i < 6; ++i) st->beta[i] = ok ? beta[i] : 0.0;
        if (I.beta_hist) {
          // coefficients in the units of the cash flow discounted to t_n
          const double to_n = 1.0 / CHK_LD(a.chk, &dtab[n]);
          for (int i = 0; i < 6; ++i)
            CHK_ST(a.chk, &I.beta_hist[(size_t)n * 6 + i],
                   ok ? (i < NB ? beta[i] * to_n : 0.0) : __longlong_as_double(0x7ff8000000000000ll));
        }
        if (I.beta_z) {  // the date's coefficients, kept for an out-of-sample pass
          for (int i = 0; i < 6; ++i) CHK_ST(a.chk, &I.beta_z[(size_t)n * 8 + i], ok ? beta[i] : 0.0);
          CHK_ST(a.chk, &I.beta_z[(size_t)n * 8 + 6], ok ? 1.0 : 0.0);
        }
        __threadfence();
        st_release_gpu(&st->ready, r + 1);
      }
    }
    __syncthreads();
  }
}

// Greeks of each (request, strike) by central differences of the scenario
// prices (the bump layout of the request's scenario table).
__global__ void greeks_kernel(const GreekOut* __restrict__ g,
                              const BwdResult* __restrict__ res, uint32_t n_out,
                              DevResult* __restrict__ out CHK_PARAM) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_out) return;
  DevResult o;
  if (form_greeks<false>(CHK_LD(chk, &g[i]), res, o CHK_ARG(chk))) CHK_ST(chk, &out[i], o);
}

cudaError_t launch_setup(BwdInstance* inst, uint32_t n_inst, cudaStream_t s CHK_PARAM) {
  if (n_inst == 0) return cudaSuccess;
  setup_kernel<<<n_inst, 128, 0, s>>>(inst, n_inst CHK_ARG(chk));
  return cudaGetLastError();
}

template <typename Real, int PPT>
static size_t bwd_dyn_bytes() {
  return (size_t)(BwdShape<Real>::kThreads / 32) * sizeof(BwdWarpBufs<Real, PPT>);
}

// dynamic shared memory above 48 KB needs the kernel's opt-in, once per device
template <typename Real, int BASIS, int PPT, int FMT>
static cudaError_t bwd_prepare() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done.load() & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(backward_kernel<Real, BASIS, PPT, FMT>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bwd_dyn_bytes<Real, PPT>());
  if (e == cudaSuccess && bit) done.fetch_or(bit);
  return e;
}

template <typename Real, int BASIS, int PPT, int FMT>
struct BwdLaunch {
  static cudaError_t run(const BwdArgs& a, int grid, cudaStream_t s) {
    const cudaError_t e = bwd_prepare<Real, BASIS, PPT, FMT>();
    if (e != cudaSuccess) return e;
    backward_kernel<Real, BASIS, PPT, FMT><<<grid, BwdShape<Real>::kThreads, bwd_dyn_bytes<Real, PPT>(), s>>>(a);
    return cudaGetLastError();
  }
};

template <typename Real, int BASIS, int PPT, int FMT>
struct BwdOccupancy {
  static int run() {
    int n = 0;
    if (bwd_prepare<Real, BASIS, PPT, FMT>() != cudaSuccess) return 1;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
               &n, backward_kernel<Real, BASIS, PPT, FMT>, BwdShape<Real>::kThreads,
               bwd_dyn_bytes<Real, PPT>()) == cudaSuccess ? n : 1;
  }
};

// F<Real, BASIS, PPT, FMT>::run(args...) for a (basis, store format)
template <template <typename, int, int, int> class F, typename Real, int PPT, typename... A>
static auto by_basis_format(int basis, int fmt, A... args) {
  if (basis == kBasisSV2) {
    if (fmt == kStoreF16) return F<Real, kBasisSV2, PPT, kStoreF16>::run(args...);
    if (fmt == kStoreBF16) return F<Real, kBasisSV2, PPT, kStoreBF16>::run(args...);
    return F<Real, kBasisSV2, PPT, kStoreNative>::run(args...);
  }
  if (fmt == kStoreF16) return F<Real, kBasisS2, PPT, kStoreF16>::run(args...);
  if (fmt == kStoreBF16) return F<Real, kBasisS2, PPT, kStoreBF16>::run(args...);
  return F<Real, kBasisS2, PPT, kStoreNative>::run(args...);
}

// ... for a (precision, basis, paths per thread, store format)
template <template <typename, int, int, int> class F, typename... A>
static auto by_variant(int precision, int basis, int ppt, int fmt, A... args) {
  if (precision == kPrecFP64)
    return ppt == 2 ? by_basis_format<F, double, 2>(basis, fmt, args...)
                    : by_basis_format<F, double, 4>(basis, fmt, args...);
  if (precision == kPrecDF)
    return ppt == 2 ? by_basis_format<F, df, 2>(basis, fmt, args...)
                    : by_basis_format<F, df, 4>(basis, fmt, args...);
  return ppt == 4 ? by_basis_format<F, float, 4>(basis, fmt, args...)
                  : by_basis_format<F, float, 8>(basis, fmt, args...);
}

// Paths per thread in a sub-tile: 2 or 4 for double and float pairs, 4 or 8
// for float.
int backward_ppt_default(int precision) { return precision == kPrecMixed ? 8 : 4; }
bool backward_ppt_valid(int precision, int ppt) {
  return precision == kPrecMixed ? (ppt == 4 || ppt == 8) : (ppt == 2 || ppt == 4);
}

cudaError_t launch_backward(const BwdArgs& a, int precision, int basis, int ppt, int grid,
                            cudaStream_t s) {
  if (a.total_jobs == 0) return cudaSuccess;
  if (!backward_ppt_valid(precision, ppt)) return cudaErrorInvalidValue;
  if (a.store_fmt < kStoreNative || a.store_fmt > kStoreBF16) return cudaErrorInvalidValue;
  return by_variant<BwdLaunch>(precision, basis, ppt, a.store_fmt, a, grid, s);
}

int backward_occupancy(int precision, int basis, int ppt, int fmt) {
  if (!backward_ppt_valid(precision, ppt)) return 1;
  return by_variant<BwdOccupancy>(precision, basis, ppt, fmt);
}

cudaError_t launch_greeks(const GreekOut* g, const BwdResult* res, uint32_t n_out,
                          DevResult* out, cudaStream_t s CHK_PARAM) {
  if (n_out == 0) return cudaSuccess;
  greeks_kernel<<<(n_out + 127) / 128, 128, 0, s>>>(g, res, n_out, out CHK_ARG(chk));
  return cudaGetLastError();
}

}  // namespace lsmc
