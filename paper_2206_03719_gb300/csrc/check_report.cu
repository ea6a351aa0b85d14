// check_report.cu -- the error word of the checked build (LSMC_CHECKED) and
// lsmc_check_report.  Every kernel of a checked build records its first
// access outside the byte ranges it was given here: the error code and the
// source line of the access (checked.cuh).
#include <cuda_runtime.h>

#include "../../include/lsmc.h"
#include "kernels.h"

#ifdef LSMC_CHECKED
namespace {
// [0]: kDevErrBadIndex once an access fell outside its ranges, [1]: its line
static __device__ uint32_t g_check[2];
}  // namespace

namespace lsmc {
int check_word(uint32_t** err, uint32_t** info) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_check) != cudaSuccess || !p) return LSMC_ECUDA;
  *err = (uint32_t*)p;
  *info = (uint32_t*)p + 1;
  return LSMC_OK;
}
}  // namespace lsmc
#endif

extern "C" int lsmc_check_report(uint32_t* code, uint32_t* line, int32_t reset) {
#ifdef LSMC_CHECKED
  if (!code || !line) return LSMC_EINVAL;
  uint32_t h[2] = {0, 0};
  if (cudaMemcpyFromSymbol(h, g_check, sizeof(h)) != cudaSuccess) return LSMC_ECUDA;
  *code = h[0];
  *line = h[1];
  if (reset) {
    const uint32_t z[2] = {0, 0};
    if (cudaMemcpyToSymbol(g_check, z, sizeof(z)) != cudaSuccess) return LSMC_ECUDA;
  }
  return LSMC_OK;
#else
  (void)code;
  (void)line;
  (void)reset;
  return LSMC_ENOTIMPL;
#endif
}
