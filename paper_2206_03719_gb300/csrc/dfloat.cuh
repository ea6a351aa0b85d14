// dfloat.cuh -- unevaluated pairs of floats ("double-float", hi + lo with
// |lo| <= ulp(hi) / 2): about 48 significant bits computed on the FP32
// pipes.  On a GB300 the FP64 pipe issues at about 1/64 of the FP32 rate, so
// this arithmetic carries the Longstaff-Schwartz path at close to double
// precision for a fraction of the cost of native double.
//
// Algorithms: Knuth's two-sum and Dekker's fast two-sum for additions,
// the FMA-based exact product for multiplications (as in Hida, Li and
// Bailey's double-double library), residual corrections for division and
// square root.  exp, log and the normal quantile are in df_math.cuh.
#pragma once

#include <cuda_runtime.h>

namespace lsmc {

struct df;
__device__ df df_abs(df a);
__device__ df df_max(df a, df b);
__device__ df df_fma(df a, df b, df c);

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  // exact split of a double into its top 24 bits and the next 24 (explicit:
  // a double never turns into a pair, or back, without being asked to)
  __host__ __device__ constexpr explicit df(double d)
      : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr explicit df(int i) : hi((float)i), lo(0.0f) {}
  __host__ __device__ explicit operator double() const {
    return (double)hi + (double)lo;
  }
  // found only by argument-dependent lookup, so these never hide the float
  // and double overloads for code that calls fabs, fmax or fma on scalars
  friend __device__ __forceinline__ df fabs(df a) { return df_abs(a); }
  friend __device__ __forceinline__ df fmax(df a, df b) { return df_max(a, b); }
  friend __device__ __forceinline__ df fma(df a, df b, df c) { return df_fma(a, b, c); }
};

__device__ __forceinline__ df quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df(p, __fmaf_rn(a, b, -p));
}

__device__ __forceinline__ df operator+(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.lo, p.lo);
  e = __fmaf_rn(a.lo, b.hi, e);
  return quick_two_sum(p.hi, e);
}

__device__ __forceinline__ df mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  return quick_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// a / b: q1 = a.hi r with r ~ 1 / b.hi (approximate reciprocal and one
// Newton step), then two corrections from the residuals a - q b, each
// formed exactly with the FMA product (Karp and Markstein's scheme)
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ df operator/(df a, df b) {
  const float r0 = rcp_approx(b.hi);
  const float r = __fmaf_rn(r0, __fmaf_rn(-b.hi, r0, 1.0f), r0);
  const float q1 = __fmul_rn(a.hi, r);
  const df p1 = two_prod(q1, b.hi);
  // a.hi - p1.hi is exact (the two agree to a few ulps)
  const df R = two_sum(__fsub_rn(a.hi, p1.hi),
                       __fmaf_rn(-q1, b.lo, __fsub_rn(a.lo, p1.lo)));
  const float q2 = __fmul_rn(R.hi, r);
  const df p2 = two_prod(q2, b.hi);
  const df s = two_sum(R.hi, -p2.hi);
  const float R2 = __fadd_rn(s.hi, __fadd_rn(s.lo, __fsub_rn(R.lo, __fmaf_rn(q2, b.lo, p2.lo))));
  const float q3 = __fmul_rn(R2, r);
  const df q = quick_two_sum(q1, q2);
  return quick_two_sum(q.hi, __fadd_rn(q.lo, q3));
}

__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ df& operator*=(df& a, df b) { return a = a * b; }

__device__ __forceinline__ bool operator<(df a, df b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool operator>(df a, df b) { return b < a; }
__device__ __forceinline__ bool operator<=(df a, df b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(df a, df b) { return !(a < b); }

__device__ __forceinline__ df df_abs(df a) { return a.hi < 0.0f ? -a : a; }
__device__ __forceinline__ df df_max(df a, df b) { return a < b ? b : a; }
__device__ __forceinline__ df df_fma(df a, df b, df c) { return a * b + c; }

// ---- cheaper forms for inner loops ---------------------------------------
// Product without the final renormalisation: hi is the float product, lo
// carries the rest unnormalised (|lo| a few ulps of hi).  Fine as an input
// to further products and sums.
__device__ __forceinline__ df mul_nr(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df(p, e);
}

// Sum without cancellation guarantees (Dekker's "sloppy" addition): exact
// two-sum of the high parts, low parts added; accurate unless a ~ -b.
__device__ __forceinline__ df add_sloppy(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

// Running sum of pairs: two-sum of the high parts, the low parts collected
// unnormalised (renormalise with quick_two_sum before using the total).
__device__ __forceinline__ void acc_pair(df& s, df t) {
  const df h = two_sum(s.hi, t.hi);
  s.hi = h.hi;
  s.lo = __fadd_rn(s.lo, __fadd_rn(h.lo, t.lo));
}

// x * 2^k, exact
__device__ __forceinline__ df ldexp_df(df a, int k) {
  return df(ldexpf(a.hi, k), ldexpf(a.lo, k));
}

__device__ __forceinline__ df sqrt_df(df a) {
  if (!(a.hi > 0.0f)) return df(0.0f, 0.0f);
  // y ~ sqrt(a.hi) from the approximate reciprocal square root, then
  // y + (a - y^2) / (2 y) with a - y^2 formed by one FMA (Karp and Markstein)
  const float x = rsqrtf(a.hi);
  const float y = __fmul_rn(a.hi, x);
  const float e = __fadd_rn(__fmaf_rn(-y, y, a.hi), a.lo);
  return quick_two_sum(y, __fmul_rn(e, __fmul_rn(x, 0.5f)));
}

}  // namespace lsmc
