// device_common.cuh -- counter-based random inputs (Philox4x32-10), uniform
// grids, the normal quantiles of single and double precision with the
// double-precision logarithm they use, and the synchronisation primitives
// shared by the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "quantile_f32.h"
#include "quantile_f64.h"

namespace lsmc {

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64-bit
// multiplies and an xor-permute, the key advancing by the Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// The same generator with the round keys given: rk[2r], rk[2r + 1] = the
// key advanced r times.  When every thread of a launch draws under one key,
// the round keys are kernel parameters, so each xor takes its key from the
// parameter bank and the key schedule costs no instruction.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t (&rk)[20]) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ rk[2 * round], lo1, hi0 ^ c.w ^ rk[2 * round + 1], lo0);
  }
  return c;
}

// (m + 1/2) 2^-52, m = top 52 bits of (hi:lo): exact, in (0, 1).
__device__ __forceinline__ double uniform52(uint32_t hi, uint32_t lo) {
  const unsigned long long m =
      ((unsigned long long)hi << 20) | (unsigned long long)(lo >> 12);
  return __fma_rn(__ull2double_rn(m), 0x1p-52, 0x1p-53);
}

// (m + 1/2) 2^-23, m = top 23 bits of w: exact, in (0, 1).
__device__ __forceinline__ float uniform23(uint32_t w) {
  return __fmaf_rn(__uint2float_rn(w >> 9), 0x1p-23f, 0x1p-24f);
}

// Standard normal quantile of a point u of the 23-bit grid (omu = 1 - u,
// exact): with x = 2u - 1 and w = -log(4 u (1 - u)), Phi^-1(u) is x times a
// smooth function of w (Giles' transformation of erfinv): a degree-8
// polynomial in w - 2.5 for w < 5, in sqrt(w) - 3 beyond (the tails, about
// 0.3% of the draws).  Coefficients: quantile_f32.h (gen_quantile_f32.py).
// Within 1e-6 of the exact quantile, max(1, |z|) relative, on every grid
// point; about 15 instructions against the library quantile's longer,
// branchier sequence.
__device__ __forceinline__ float norm_quantile_f32(float u, float omu) {
  const float lg = __log2f(__fmul_rn(u, omu));        // log2(u (1 - u))
  const float t = __fmaf_rn(lg, kQfNegLn2, kQfShift);  // w - 2.5
  const float x = __fsub_rn(u, omu);                   // 2u - 1
  float r;
  if (t < kQfSplit) {
    r = __fmaf_rn(kQfP8, t, kQfP7);
    r = __fmaf_rn(r, t, kQfP6);
    r = __fmaf_rn(r, t, kQfP5);
    r = __fmaf_rn(r, t, kQfP4);
    r = __fmaf_rn(r, t, kQfP3);
    r = __fmaf_rn(r, t, kQfP2);
    r = __fmaf_rn(r, t, kQfP1);
    r = __fmaf_rn(r, t, kQfP0);
  } else {
    float q;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(q) : "f"(__fadd_rn(t, 2.5f)));
    const float sv = __fsub_rn(q, 3.0f);
    r = __fmaf_rn(kQfQ8, sv, kQfQ7);
    r = __fmaf_rn(r, sv, kQfQ6);
    r = __fmaf_rn(r, sv, kQfQ5);
    r = __fmaf_rn(r, sv, kQfQ4);
    r = __fmaf_rn(r, sv, kQfQ3);
    r = __fmaf_rn(r, sv, kQfQ2);
    r = __fmaf_rn(r, sv, kQfQ1);
    r = __fmaf_rn(r, sv, kQfQ0);
  }
  return __fmul_rn(x, r);
}

// log(a) in double for a normal, finite, positive a (Tang's table-driven
// reduction, tables in quantile_f64.h): a = 2^e m, m in [1, 2),
// j = round(128 (m - 1)), t = m c_j - 1 by one fused multiply-add
// (|t| < 0.004), log a = e ln2 - log c_j + log1p(t), log1p by its Taylor
// series to t^7.  About 15 FP64 operations; other arguments (zero,
// subnormal, infinite, NaN, negative) go to CUDA's log.  Near a = 1 the
// ln2 terms cancel exactly and the result keeps full relative accuracy.
__device__ __forceinline__ double log_f64(double a) {
  const long long bits = __double_as_longlong(a);
  if (bits < 0x0010000000000000ll || bits >= 0x7ff0000000000000ll) return log(a);
  const double e = (double)((int)(bits >> 52) - 1023);
  const double m = __longlong_as_double((bits & 0x000fffffffffffffll) | 0x3ff0000000000000ll);
  const int j = ((int)((bits >> 44) & 0xff) + 1) >> 1;  // nearest integer to 128 (m - 1)
  const double t = fma(m, __ldg(&kLogRecip[j]), -1.0);
  // log1p(t) = t + t^2 q(t), q = -1/2 + t/3 - t^2/4 + t^3/5 - t^4/6 + t^5/7
  double q = fma(t, 1.0 / 7.0, -1.0 / 6.0);
  q = fma(q, t, 1.0 / 5.0);
  q = fma(q, t, -1.0 / 4.0);
  q = fma(q, t, 1.0 / 3.0);
  q = fma(q, t, -0.5);
  const double lp = fma(t * t, q, t);
  const double hi = fma(e, kLn2Hi, __ldg(&kLogNegHi[j]));  // e ln2_hi is exact
  return hi + fma(e, kLn2Lo, __ldg(&kLogNegLo[j]) + lp);
}

// Standard normal quantile of a point u of the 52-bit grid (omu = 1 - u,
// exact) in double: Giles' transformation as in norm_quantile_f32, with
// w = -log(4 u (1 - u)) by log_f64 and polynomials of degree 23 in w - 3.125
// for w < 6.25, 18 and 16 in sqrt(w) beyond (the tails, about 0.1% of the
// draws); coefficients in quantile_f64.h (gen_quantile_f64.py), each
// polynomial within 2.5e-16 of the exact quotient.
__device__ __forceinline__ double norm_quantile_f64(double u, double omu) {
  const double w = -log_f64(4.0 * (u * omu));
  const double x = u - omu;  // 2u - 1
  double r;
  if (w < kQdSplitW) {
    r = qd_central(w - kQdCentreW);
  } else {
    const double s = sqrt(w);
    r = s < kQdSplitS ? qd_tail1(s - kQdCentreS1) : qd_tail2(s - kQdCentreS2);
  }
  return x * r;
}

// Random inputs of one path step from one Philox block: the uniform U_V,
// 1 - U_V (exact in both grids), Z_V = Phi^-1(U_V) and Z_X.  The float-pair
// specialisation is in df_math.cuh and uses the tables t stages in shared
// memory; the others ignore t.
struct DfTables;
template <typename Real> struct Draw;
template <> struct Draw<double> {
  // U_V, Z_V from words (0, 1); Z_X from words (2, 3)
  __device__ __forceinline__ static void make(uint4 w, double& u, double& omu, double& zV,
                                              double& zX, const DfTables*) {
    u = uniform52(w.x, w.y);
    omu = 1.0 - u;
    zV = norm_quantile_f64(u, omu);
    const double uX = uniform52(w.z, w.w);
    zX = norm_quantile_f64(uX, 1.0 - uX);
  }
};
template <> struct Draw<float> {
  // U_V from word 0 and Z_X from word 2: the top 23 bits of the words the
  // double-precision grid reads first, so both precisions see one stream
  __device__ __forceinline__ static void make(uint4 w, float& u, float& omu, float& zV,
                                              float& zX, const DfTables*) {
    u = uniform23(w.x);
    omu = 1.0f - u;
    zV = norm_quantile_f32(u, omu);
    const float uX = uniform23(w.z);
    zX = norm_quantile_f32(uX, 1.0f - uX);
  }
};

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
  return *(const volatile uint32_t*)p;
}

// L2-coherent loads of data other CTAs wrote during this launch
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ df ld_cg(const df* p) {
  const float2 v = __ldcg((const float2*)p);
  return df(v.x, v.y);
}

}  // namespace lsmc
