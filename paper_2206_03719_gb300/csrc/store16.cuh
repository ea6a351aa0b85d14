// store16.cuh -- the element types of the path store and the conversions
// between them and the working precision.
//
// The path store holds, per path group and date, exp(x) (x = log(S / S0))
// and the variance.  Besides the working precision it can be IEEE binary16
// or bfloat16 (the paper's study of reduced data types, Sec. 4.2 and
// Table 4, applied to the stored paths only: every step is still computed in
// the working precision, and a stored value is rounded once, to nearest with
// ties to even, when it is written and widened exactly when it is read).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "dfloat.cuh"
#include "plan.h"

namespace lsmc {

// element type of the store for a working precision and a store format
template <typename Real, int FMT> struct StoreElem { using type = Real; };
template <typename Real> struct StoreElem<Real, kStoreF16> { using type = __half; };
template <typename Real> struct StoreElem<Real, kStoreBF16> { using type = __nv_bfloat16; };

// ---- narrowing: round to nearest, ties to even ------------------------------
template <typename St, typename Real> __device__ __forceinline__ St narrow(Real v);

template <> __device__ __forceinline__ double narrow<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float narrow<float, float>(float v) { return v; }
template <> __device__ __forceinline__ df narrow<df, df>(df v) { return v; }

template <> __device__ __forceinline__ __half narrow<__half, double>(double v) {
  return __double2half(v);
}
template <> __device__ __forceinline__ __half narrow<__half, float>(float v) {
  return __float2half_rn(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 narrow<__nv_bfloat16, double>(double v) {
  return __double2bfloat16(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 narrow<__nv_bfloat16, float>(float v) {
  return __float2bfloat16_rn(v);
}

// A float pair a = hi + lo (|lo| at most half a unit in the last place of hi)
// rounded as one number.  Every value of the narrow format and every midpoint
// between two neighbours is a float, so rounding hi alone is right unless hi
// is such a midpoint; then lo decides (away from zero when lo has hi's sign,
// towards zero when it has the other sign, ties to even when lo = 0).
template <> __device__ __forceinline__ __half narrow<__half, df>(df a) {
  const __half t = __float2half_rz(a.hi);  // the neighbour towards zero
  const __half u = __ushort_as_half((unsigned short)(__half_as_ushort(t) + 1u));
  const float mid = 0.5f * (__half2float(t) + __half2float(u));  // exact
  if (a.hi == mid && a.lo != 0.0f) return ((a.lo > 0.0f) == (a.hi > 0.0f)) ? u : t;
  return __float2half_rn(a.hi);
}
template <> __device__ __forceinline__ __nv_bfloat16 narrow<__nv_bfloat16, df>(df a) {
  const __nv_bfloat16 t = __float2bfloat16_rz(a.hi);
  const __nv_bfloat16 u =
      __ushort_as_bfloat16((unsigned short)(__bfloat16_as_ushort(t) + 1u));
  const float mid = 0.5f * (__bfloat162float(t) + __bfloat162float(u));  // exact
  if (a.hi == mid && a.lo != 0.0f) return ((a.lo > 0.0f) == (a.hi > 0.0f)) ? u : t;
  return __float2bfloat16_rn(a.hi);
}

// ---- widening: exact --------------------------------------------------------
template <typename Real> __device__ __forceinline__ Real widen(Real v) { return v; }
template <typename Real> __device__ __forceinline__ Real widen(__half v);
template <typename Real> __device__ __forceinline__ Real widen(__nv_bfloat16 v);
template <> __device__ __forceinline__ double widen<double>(__half v) {
  return (double)__half2float(v);
}
template <> __device__ __forceinline__ float widen<float>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ df widen<df>(__half v) { return df(__half2float(v), 0.0f); }
template <> __device__ __forceinline__ double widen<double>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}
template <> __device__ __forceinline__ float widen<float>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <> __device__ __forceinline__ df widen<df>(__nv_bfloat16 v) {
  return df(__bfloat162float(v), 0.0f);
}

// Reading rows: raw elements (the working precision, or the 16 bits as an
// unsigned short) loaded first and widened afterwards, so a thread's loads
// are all issued before the first conversion waits on one.
template <typename Real, int FMT> struct RowRead {
  using raw = Real;
  __device__ __forceinline__ static Real widen(raw r) { return r; }
};
template <typename Real> struct RowRead<Real, kStoreF16> {
  using raw = unsigned short;
  __device__ __forceinline__ static Real widen(raw r) {
    return lsmc::widen<Real>(__ushort_as_half(r));
  }
};
template <typename Real> struct RowRead<Real, kStoreBF16> {
  using raw = unsigned short;
  __device__ __forceinline__ static Real widen(raw r) {
    return lsmc::widen<Real>(__ushort_as_bfloat16(r));
  }
};

}  // namespace lsmc
