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

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

}  // namespace
}  // namespace lsmc
