// exercise.cuh -- payoff, exercise test and the small arithmetic helpers
// shared by the backward induction (backward.cu) and the out-of-sample
// pricing pass (oos.cu), so both take every exercise decision with the same
// operations in the same order.
#pragma once

#include <cmath>
#include <type_traits>

#include "dfloat.cuh"
#include "plan.h"

namespace lsmc {
namespace {

__device__ __forceinline__ double payoff_d(int type, double K, double S) {
  const double h = type == kPut ? K - S : S - K;
  return h > 0.0 ? h : 0.0;
}

template <typename Real>
__device__ __forceinline__ Real payoff(int type, Real K, Real S) {
  const Real h = type == kPut ? K - S : S - K;
  return h > (Real)0 ? h : (Real)0;
}

// Inner-loop arithmetic: plain operators for float and double, the cheaper
// unnormalised forms for float pairs.
template <typename R> __device__ __forceinline__ R qmul(R a, R b) { return a * b; }
template <> __device__ __forceinline__ df qmul<df>(df a, df b) { return mul_nr(a, b); }
template <typename R> __device__ __forceinline__ void qacc(R& s, R t) { s += t; }
template <> __device__ __forceinline__ void qacc<df>(df& s, df t) { acc_pair(s, t); }
// a * b + c
template <typename R> __device__ __forceinline__ R qfma(R a, R b, R c) { return fma(a, b, c); }
template <> __device__ __forceinline__ df qfma<df>(df a, df b, df c) {
  return add_sloppy(mul_nr(a, b), c);
}
template <typename R> __device__ __forceinline__ R qsub(R a, R b) { return a - b; }
template <> __device__ __forceinline__ df qsub<df>(df a, df b) { return add_sloppy(a, -b); }
// payoff without the max: put K - S, call S - K
template <typename R>
__device__ __forceinline__ R intrinsic(int type, R K, R S) {
  return type == kPut ? qsub(K, S) : qsub(S, K);
}

// In the money (payoff strictly positive) without forming the payoff: for
// positive doubles the bit patterns order like the values, so the test runs
// on the integer pipe instead of the narrow FP64 one.
template <typename R>
__device__ __forceinline__ bool in_money(int type, R K, R S) {
  return type == kPut ? S < K : K < S;
}
template <>
__device__ __forceinline__ bool in_money<double>(int type, double K, double S) {
  const long long s = __double_as_longlong(S), k = __double_as_longlong(K);
  return type == kPut ? s < k : k < s;
}

// Exercise decision (discounted payoff hd against fitted value c) and the
// near-tie flag (|hd - c| within about 1e-10 of max(|c|, hd)).
template <typename R>
__device__ __forceinline__ void decide(R hd, R c, bool& exercise, bool& tie) {
  tie = fabs(hd - c) <= (R)kTieRel * fmax(fabs(c), hd);
  exercise = hd > c;
}
template <>
__device__ __forceinline__ void decide<double>(double hd, double c, bool& exercise, bool& tie) {
  // one FP64 subtraction; sign and exponents compared as integers
  // (2^-33 = 1.16e-10 relative)
  const double d = hd - c;
  const long long bd = __double_as_longlong(d);
  exercise = bd > 0;
  const int ed = (int)((bd >> 52) & 0x7ff);
  const int ec = (int)((__double_as_longlong(c) >> 52) & 0x7ff);
  const int eh = (int)((__double_as_longlong(hd) >> 52) & 0x7ff);
  tie = ed + 33 <= max(ec, eh);
}
template <>
__device__ __forceinline__ void decide<df>(df hd, df c, bool& exercise, bool& tie) {
  const df d = add_sloppy(hd, -c);
  tie = fabsf(d.hi) <= (float)kTieRel * fmaxf(fabsf(c.hi), hd.hi);
  exercise = d.hi > 0.0f || (d.hi == 0.0f && d.lo > 0.0f);
}

// The in-the-money test of a stored value e at a date with S multiplier s1,
// RN(s1 e) < K (put) or RN(s1 e) > K (call), as one comparison of e against
// a threshold: RN(s1 e) does not decrease as e grows, so for a put the
// values in the money are those below the smallest e with RN(s1 e) >= K,
// and for a call those above the largest e with RN(s1 e) <= K.
// The start K / s1 is within a few units in the last place of the answer;
// the walks are bounded all the same (s1 > 0 and K > 0 are finite).
__device__ double itm_threshold(int type, double s1, double K) {
  double e = K / s1;
  if (type == kPut) {
    for (int i = 0; i < 64 && s1 * e >= K; ++i) e = nextafter(e, 0.0);  // RN(s1 e) < K
    e = nextafter(e, HUGE_VAL);  // the smallest e with RN(s1 e) >= K
    for (int i = 0; i < 64 && s1 * e < K; ++i) e = nextafter(e, HUGE_VAL);
  } else {
    for (int i = 0; i < 64 && s1 * e <= K; ++i) e = nextafter(e, HUGE_VAL);  // RN(s1 e) > K
    e = nextafter(e, 0.0);  // the largest e with RN(s1 e) <= K
    for (int i = 0; i < 64 && s1 * e > K; ++i) e = nextafter(e, 0.0);
  }
  return e;
}

// the bits of a stored in-the-money threshold (double only; the other
// precisions test the product itself)
__device__ __forceinline__ long long threshold_bits(double t) { return __double_as_longlong(t); }
__device__ __forceinline__ long long threshold_bits(float) { return 0; }
__device__ __forceinline__ long long threshold_bits(df) { return 0; }

// in_money(type, K, RN(s e)); for double through the threshold's bits
template <typename R>
__device__ __forceinline__ bool itm_test(int type, R K, R s, R e, long long) {
  return in_money<R>(type, K, s * e);  // normalised: the comparison reads hi first
}
template <>
__device__ __forceinline__ bool itm_test<double>(int type, double, double, double e,
                                                 long long thr) {
  const long long eb = __double_as_longlong(e);
  return type == kPut ? eb < thr : eb > thr;
}

// ---- float screen of the exercise test ---------------------------------------
// The exercise test hd > c (hd the discounted payoff, c the fitted
// continuation value) costs about a dozen operations of the working
// precision per in-the-money path: FP64 ones, on GB300's narrow FP64 pipe,
// or float-pair ones of ten FP32 instructions each.  Almost every decision
// is far from its threshold, so it is first taken in float, with a bound on
// the float result's error; only when |hd - c| is within that bound (and
// always when the decision could be a near tie) does the caller run the test
// in the working precision.  Decisions, near-tie counts and cash flows are
// therefore exactly those of the test itself.
//
// Error bound.  The float inputs carry relative errors of at most 2^-23 (S,
// v) and 2^-24 (constants), so x = S/K - 1 and w = v/theta - 1 are off by at
// most 3.6e-7 (1 + |x|) and 2.4e-7 (1 + |w|); every monomial of the basis is
// at most M^2 with M = 1 + |x| + |w|, and moves by at most 7.2e-7 M^2; the
// coefficients' rounding and the six rounded operations add 4.2e-7 B M^2
// (B = sum |beta_i|): |c_float - c| <= 1.2e-6 B M^2.  The payoff
// h = K - S is off by at most 2.5e-7 (2K + |h|), so |hd_float - hd| <=
// 5e-7 (K d + |hd|).  The screen decides only when |hd - c| exceeds
// 3.2e-5 (B M^2 + K d + |hd|), 25 times the bound, which also exceeds the
// near-tie distance 1e-10 max(|c|, hd) by far.
struct ScreenConsts {
  float b[6];      // coefficients (zero where the basis has fewer)
  float s, K, invK, invTh, d;  // S multiplier of the row value, strike, 1/K, 1/theta, discount
  float B;         // sum of |b_i|
};
static_assert(sizeof(ScreenConsts) == kScreenBytes, "table layout");

// float value of a double within 2^-23 relative (the mantissa truncated,
// integer operations only): 0 below float's normal range, infinity above
__device__ __forceinline__ float approx_float(double x) {
  const unsigned long long bits = __double_as_longlong(x);
  const unsigned hi = (unsigned)(bits >> 32);
  const int e = (int)((hi >> 20) & 0x7ffu);
  if (e < 1023 - 126) return 0.0f;
  const unsigned sign = hi & 0x80000000u;
  if (e > 1023 + 127) return __uint_as_float(sign | 0x7f800000u);
  const unsigned mag = (unsigned)((bits & 0x7fffffffffffffffull) >> 29) - ((1023u - 127u) << 23);
  return __uint_as_float(sign | mag);
}
__device__ __forceinline__ float approx_float(df x) { return x.hi; }
__device__ __forceinline__ float approx_float(float x) { return x; }

// 1: exercise, 0: continue, 2: undecided.  e: the row value (S = s e) and v
// the variance of an in-the-money path.
template <int BASIS>
__device__ __forceinline__ int exercise_screen(const ScreenConsts& q, int type, float e, float v) {
  const float S = __fmul_rn(q.s, e);
  const float x = __fmaf_rn(S, q.invK, -1.0f);
  float c = __fmaf_rn(__fmaf_rn(q.b[2], x, q.b[1]), x, q.b[0]);
  float M = 1.0f + fabsf(x);
  if (BASIS == kBasisSV2) {
    const float w = __fmaf_rn(v, q.invTh, -1.0f);
    c = __fmaf_rn(__fmaf_rn(q.b[5], w, __fmaf_rn(q.b[4], x, q.b[3])), w, c);
    M += fabsf(w);
  }
  const float h = type == kPut ? __fsub_rn(q.K, S) : __fsub_rn(S, q.K);
  const float hd = __fmul_rn(h, q.d);
  const float bound = 3.2e-5f * (q.B * M * M + q.K * q.d + fabsf(hd));
  const float diff = __fsub_rn(hd, c);
  return diff > bound ? 1 : (diff < -bound ? 0 : 2);
}

// ScreenConsts from the working-precision values (b: the basis's
// coefficients, 3 or 6)
template <int BASIS, typename Real>
__device__ __forceinline__ void make_screen(ScreenConsts& q, const Real* b, Real s, Real K,
                                            Real invK, Real invTh, Real d) {
  float B = 0.0f;
  for (int i = 0; i < 6; ++i) {
    q.b[i] = (i < 3 || BASIS == kBasisSV2) ? (float)(double)b[i] : 0.0f;
    B += fabsf(q.b[i]);
  }
  q.B = B;
  q.s = (float)(double)s;
  q.K = (float)(double)K;
  q.invK = (float)(double)invK;
  q.invTh = (float)(double)invTh;
  q.d = (float)(double)d;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

}  // namespace
}  // namespace lsmc
