// checked.cuh -- global-memory accesses of the kernels, tested against the
// launch's byte ranges in the checked build (LSMC_CHECKED) and plain in the
// ordinary one.  The checked build is the library's own bounds checker: a
// kernel's access outside every range it was given records an error word and
// the source line, and is skipped (a load yields zero) -- no trap, no fault.
//
//   CHK_LD(c, p)     value at p
//   CHK_ST(c, p, v)  *p = v
//   CHK_OK(c, p, n)  the n bytes at p lie inside a range (guard other accesses:
//                    atomics, cache-hinted loads, vector accesses)
// c is the launch's CheckRanges; the ordinary build never evaluates it.
#pragma once

#include <cstdint>

#include "plan.h"

namespace lsmc {

#ifdef LSMC_CHECKED
__device__ __forceinline__ bool chk_ok(const CheckRanges& c, const void* p, size_t bytes,
                                       int line) {
  const unsigned long long a = (unsigned long long)p, b = a + bytes;
  for (uint32_t i = 0; i < c.n && i < (uint32_t)kMaxRanges; ++i)
    if (a >= c.lo[i] && b <= c.hi[i] && b >= a) return true;
  if (c.err && atomicCAS(c.err, 0u, kDevErrBadIndex) == 0u && c.info)
    atomicExch(c.info, (uint32_t)line);
  return false;
}
template <typename T>
__device__ __forceinline__ T chk_ld(const CheckRanges& c, const T* p, int line) {
  return chk_ok(c, p, sizeof(T), line) ? *p : T();
}
template <typename T, typename V>
__device__ __forceinline__ void chk_st(const CheckRanges& c, T* p, V v, int line) {
  if (chk_ok(c, p, sizeof(T), line)) *p = v;
}
#define CHK_LD(c, p) ::lsmc::chk_ld((c), (p), __LINE__)
#define CHK_ST(c, p, v) ::lsmc::chk_st((c), (p), (v), __LINE__)
#define CHK_OK(c, p, n) ::lsmc::chk_ok((c), (p), (n), __LINE__)
#else
#define CHK_LD(c, p) (*(p))
#define CHK_ST(c, p, v) (*(p) = (v))
#define CHK_OK(c, p, n) true
#endif

}  // namespace lsmc
