// df_math.cuh -- exp, log and the standard normal quantile on float pairs,
// all on the FP32 pipes.  The constant tables (df_tables.h, written by
// gen_df_tables.py) are staged in shared memory by the kernels that use
// them (load_df_tables), because the table index differs from lane to lane.
#pragma once

#include <cstdint>

#include "dfloat.cuh"
#include "df_tables.h"

namespace lsmc {

struct DfTables {
  float2 exp2[kExpTab];                          // 2^(j / kExpTab)
  float2 qpair[kQPair][kQIntervals];             // G polynomials, pair part
  float qflt[kQDegree + 1 - kQPair][kQIntervals];  // G polynomials, float part
  float qcen[kQIntervals];                       // interval centres
};

// Copy the tables into shared memory; the caller synchronises the block.
__device__ __forceinline__ void load_df_tables(DfTables* t) {
  for (int i = threadIdx.x; i < kExpTab; i += blockDim.x) t->exp2[i] = kExp2Frac[i];
  for (int i = threadIdx.x; i < kQPair * kQIntervals; i += blockDim.x)
    (&t->qpair[0][0])[i] = (&kQCoefPair[0][0])[i];
  for (int i = threadIdx.x; i < (kQDegree + 1 - kQPair) * kQIntervals; i += blockDim.x)
    (&t->qflt[0][0])[i] = (&kQCoefFloat[0][0])[i];
  for (int i = threadIdx.x; i < kQIntervals; i += blockDim.x) t->qcen[i] = kQCentre[i];
}

// exp(a).  Reduction a = k L + r with L = ln 2 / kExpTab split into three
// floats (Cody and Waite: k C1 is exact, k C2 is an exact product pair), so
// |r| <= L / 2 ~ 0.0027, held to about 2^-56 absolute; then
// exp(a) = 2^n 2^(j / kExpTab) exp(r) with k = n kExpTab + j.  exp(r) - 1 = r + r^2 / 2 + r^3 (1/6 + r / 24 + r^2 / 120):
// r^2 is an exact product pair, the cubic tail (< 4e-9) is summed in float.
__device__ __forceinline__ df exp_df(df a, const float2* tab) {
  if (a.hi > 88.0f) return df(__int_as_float(0x7f800000), 0.0f);
  if (a.hi < -87.0f) return df(0.0f, 0.0f);
  const float kf = rintf(__fmul_rn(a.hi, kExpInvL));
  const int k = (int)kf;
  const float t1 = __fmaf_rn(-kf, kExpC1, a.hi);  // exact (Sterbenz)
  const df p2 = two_prod(kf, kExpC2);
  // a.lo (up to half an ulp of a.hi, 2e-6 at |a| = 60) is added by a two-sum:
  // folded into the low word in float it would cost up to 2^-43 absolute
  const df d = two_sum(t1, -p2.hi);
  const df e0 = two_sum(d.hi, a.lo);
  const df r = quick_two_sum(
      e0.hi, __fadd_rn(e0.lo, __fsub_rn(d.lo, __fmaf_rn(kf, kExpC3, p2.lo))));
  df r2 = two_prod(r.hi, r.hi);
  r2.lo = __fmaf_rn(__fadd_rn(r.hi, r.hi), r.lo, r2.lo);
  const float tail = __fmul_rn(__fmul_rn(r2.hi, r.hi),
                               __fmaf_rn(r.hi, __fmaf_rn(r.hi, 1.0f / 120.0f, 1.0f / 24.0f),
                                         1.0f / 6.0f));
  df e = add_sloppy(r, df(__fmul_rn(r2.hi, 0.5f), __fmul_rn(r2.lo, 0.5f)));
  e.lo = __fadd_rn(e.lo, tail);
  const float2 tj = tab[k & (kExpTab - 1)];
  const df T(tj.x, tj.y);
  const df res = add_sloppy(T, mul_nr(T, e));
  // 2^n with n = floor(k / kExpTab) in [-126, 126] for |a| < 88
  const float s = __int_as_float(((k >> 7) + 127) << 23);
  static_assert(kExpTab == 128, "the shift above is log2(kExpTab)");
  return df(__fmul_rn(res.hi, s), __fmul_rn(res.lo, s));
}

// exp(x) in double, table-driven (Tang's method): k = rint(x 128 / ln 2)
// (adding 1.5 2^52 leaves k in the low mantissa bits), r = x - k ln2/128 by
// two fused multiply-adds (|r| <= ln2/256), exp(r) - 1 = r + r^2 (1/2 + r/6 +
// r^2/24 + r^3/120) (the truncated terms stay below 6e-19), and
// exp(x) = 2^(k >> 7) * 2^((k & 127)/128) (1 + (exp(r) - 1)): about 10 FP64
// operations against CUDA's exp at about 16 (measured on GB300), within one
// unit in the last place.  Outside |x| < 512 (where the final scaling by
// the exponent field could overflow or underflow) CUDA's exp.
__device__ __forceinline__ double exp_f64(double x) {
  const unsigned long long bits = __double_as_longlong(x);
  if (((bits >> 52) & 0x7ffull) >= 1023ull + 9ull) return exp(x);
  const double magic = 6755399441055744.0;  // 1.5 * 2^52
  const double t = fma(x, kExpF64InvL, magic);
  const int k = __double2loint(t);
  const double kf = t - magic;
  double r = fma(-kf, kExpF64C1, x);
  r = fma(-kf, kExpF64C2, r);
  const double q = fma(fma(fma(r, 1.0 / 120.0, 1.0 / 24.0), r, 1.0 / 6.0), r, 0.5);
  const double p = fma(r * r, q, r);
  const double T = __ldg(&kExp2F64[k & (kExpTab - 1)]);
  const double y = fma(T, p, T);
  return __longlong_as_double(__double_as_longlong(y) + ((long long)(k >> 7) << 52));
}

// log(a), a > 0: y0 = logf(a.hi), then one Newton step on exp(y) = a,
// y1 = y0 + a exp(-y0) - 1 (quadratic: the float error squared)
__device__ __forceinline__ df log_df(df a, const float2* tab) {
  if (!(a.hi > 0.0f)) return df(-__int_as_float(0x7f800000), 0.0f);
  const float y0 = logf(a.hi);
  const df t = a * exp_df(df(-y0, 0.0f), tab) - df(1.0f, 0.0f);
  return df(y0, 0.0f) + t;
}

// hi 2^-32 + l21 2^-53 (hi a 32-bit word, l21 < 2^21) as a pair: three
// exact floats (16 + 16 + 21 bits) summed without cancellation
__device__ __forceinline__ df uniform_pair(uint32_t hi, uint32_t l21) {
  const float a = __fmul_rn(__uint2float_rn(hi >> 16), 0x1p-16f);
  const float b = __fmul_rn(__uint2float_rn(hi & 0xffffu), 0x1p-32f);
  const float c = __fmul_rn(__uint2float_rn(l21), 0x1p-53f);
  return add_sloppy(two_sum(a, b), df(c, 0.0f));
}

// Standard normal quantile z = Phi^-1(p) for 0 < p <= 1/2 given as a pair
// (returns z <= 0).  z0 = normcdfinvf(p.hi) has a float's accuracy; one
// Halley step on f(z) = Phi(z) - p finishes it:
//   d = f(z0) / phi(z0) = sqrt(2 pi) (G(z0) - p exp(z0^2 / 2)),
//   z1 = z0 - d / (1 + z0 d / 2) ~ z0 - d + z0 d^2 / 2,
// with G(z) = Phi(z) exp(z^2 / 2) from the per-interval polynomials in
// x = z0 - c (exact in float, see gen_df_tables.py) and z0^2 / 2 an exact
// product pair.  The error of z0 is cubed, so z1 carries the pair precision.
__device__ __forceinline__ df normal_quantile_lower_df(df p, const DfTables* t) {
  const float z0 = normcdfinvf(p.hi);
  const float m = -z0;
  const int i = m < 0.25f ? 0 : (m < 0.5f ? 1 : min(1 + (int)(m + m), kQIntervals - 1));
  const float x = __fsub_rn(z0, t->qcen[i]);
  float g = t->qflt[kQDegree - kQPair][i];
#pragma unroll
  for (int k = kQDegree - kQPair - 1; k >= 0; --k) g = __fmaf_rn(g, x, t->qflt[k][i]);
  const float2 ct = t->qpair[kQPair - 1][i];
  df G(ct.x, __fmaf_rn(g, x, ct.y));
#pragma unroll
  for (int k = kQPair - 2; k >= 0; --k) {
    const float2 c = t->qpair[k][i];
    const df gx = two_prod(G.hi, x);
    G = add_sloppy(df(c.x, c.y), df(gx.hi, __fmaf_rn(G.lo, x, gx.lo)));
  }
  df q = two_prod(z0, z0);
  q = df(__fmul_rn(q.hi, 0.5f), __fmul_rn(q.lo, 0.5f));
  const df r = G - p * exp_df(q, t->exp2);
  constexpr double kSqrt2Pi = 2.50662827463100050241576528481104525;
  const df d = mul_nr(r, df(kSqrt2Pi));
  const float corr = __fmul_rn(__fmul_rn(z0, d.hi), __fmul_rn(d.hi, 0.5f));
  const df s = two_sum(z0, -d.hi);
  return quick_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(corr, d.lo)));
}

// The random inputs of one path step from one Philox block, as pairs:
// u = (m + 1/2) 2^-52 from words (0, 1) (the FP64 grid), 1 - u, and the two
// normal quantiles of the FP64 grid points of words (0, 1) and (2, 3).
// With M = 2m + 1 = hi 2^21 + l21 (l21 odd, < 2^21): u = hi 2^-32 + l21 2^-53
// and 1 - u = (~hi) 2^-32 + (2^21 - l21) 2^-53, both exact before pairing.
template <> struct Draw<df> {
  __device__ __forceinline__ static df quantile(uint32_t hi, uint32_t lo,
                                                const DfTables* t) {
    const uint32_t l21 = (lo >> 11) | 1u;
    const bool upper = (hi >> 31) != 0u;
    const df p = upper ? uniform_pair(~hi, 0x200000u - l21) : uniform_pair(hi, l21);
    const df z = normal_quantile_lower_df(p, t);
    return upper ? -z : z;
  }
  __device__ __forceinline__ static void make(uint4 w, df& u, df& omu, df& zV, df& zX,
                                              const DfTables* t) {
    const uint32_t l21 = (w.y >> 11) | 1u;
    u = uniform_pair(w.x, l21);
    omu = uniform_pair(~w.x, 0x200000u - l21);
    zV = quantile(w.x, w.y, t);
    zX = quantile(w.z, w.w, t);
  }
};

}  // namespace lsmc
