// kernels.h -- host-side launchers of the device kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "plan.h"

namespace lsmc {

cudaError_t launch_forward(const FwdArgs& a, int precision, int scheme, cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1,
                          uint32_t* out, size_t n, cudaStream_t s);
cudaError_t launch_draws(uint64_t seed, uint32_t stream_id, const uint32_t* path,
                         const uint32_t* step, size_t n, int precision, void* out,
                         cudaStream_t s);
cudaError_t launch_multi_max(const MultiArgs& a, int precision, int scheme, cudaStream_t s);
// the forward pass's exponential on n values of the precision
cudaError_t launch_exp(const void* x, void* y, size_t n, int precision, cudaStream_t s);
cudaError_t launch_quantile(const void* u, void* z, size_t n, int precision, cudaStream_t s);
cudaError_t launch_setup(BwdInstance* inst, uint32_t n_inst, cudaStream_t s CHK_PARAM);
cudaError_t launch_backward(const BwdArgs& a, int precision, int basis, int ppt, int grid,
                            cudaStream_t s);
// out-of-sample pricing pass over the instances' rows and its estimator
cudaError_t launch_oos(const BwdInstance* inst, uint32_t n_inst, uint32_t max_paths,
                       const BwdState* state, BwdResult* results, int precision, int basis,
                       int fmt, cudaStream_t s CHK_PARAM);
// dual upper bound of the strikes of one request (the plan's policy tables
// must be filled: after launch_oos)
cudaError_t launch_dual(const DualArgs& a, int precision, int scheme, int basis, cudaStream_t s);
cudaError_t launch_greeks(const GreekOut* g, const BwdResult* res, uint32_t n_out,
                          DevResult* out, cudaStream_t s CHK_PARAM);
// Paths per thread of a backward sub-tile (a sub-tile is kBlock * ppt
// paths): the default for a precision and whether a value is compiled for it.
int backward_ppt_default(int precision);
bool backward_ppt_valid(int precision, int ppt);
// threads per CTA of the backward pass (64 for FP64, kBlock otherwise) and
// paths per backward sub-tile
inline int backward_block(int precision) { return precision == kPrecFP64 ? 64 : kBlock; }
inline int backward_tile(int precision, int ppt) { return backward_block(precision) * ppt; }
// resident backward CTAs per SM of a kernel variant (fmt: store format)
int backward_occupancy(int precision, int basis, int ppt, int fmt);
// bytes of one working-precision value (cash flow, saved state) in a precision
inline size_t value_bytes(int precision) { return precision == kPrecMixed ? 4 : 8; }
// bytes of one element of the E/V rows in a precision and store format
inline size_t row_bytes(int precision, int fmt) {
  return fmt == kStoreNative ? value_bytes(precision) : 2;
}

}  // namespace lsmc

#include "../../include/lsmc.h"

namespace lsmc {
// Backward pass of lsmc_backward with every temporary placed in the given
// device range instead of freshly allocated memory (capi.cpp).
#ifdef LSMC_CHECKED
// device addresses of the checked build's error word (code, source line) on
// the current device (check_report.cu)
int check_word(uint32_t** err, uint32_t** info);
#endif
int backward_in_scratch(void* scratch, size_t scratch_bytes, const void* d_S, const void* d_V,
                        uint32_t P, uint32_t N, int32_t precision, const lsmc_heston* m,
                        const lsmc_contract* c, int32_t basis, double* d_out, double* d_beta,
                        uint32_t* d_nsing, cudaStream_t s);
}  // namespace lsmc
