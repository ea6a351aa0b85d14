// noalloc.cu -- lsmc_backward_noalloc: the Longstaff-Schwartz backward pass
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while another
// allocator owns the device (a framework's caching allocator, a fixed memory
// budget carved out up front), code on a latency-critical path where
// cudaMalloc/cudaFree would synchronise the device, or code that has to keep
// working when the device is nearly full.  For them this entry point keeps
// its scratch memory (job tables, per-tile partial sums, cash flows, counters)
// in one file-scope array of kScratchBytes that the library carries in device
// memory; the caller still passes the paths and the output buffers.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lsmc.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB per device

// Every device that loads this library holds this array until the process
// exits.  In host code the name is only a host-side stand-in: its device
// address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LSMC_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return LSMC_ENODEV;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return LSMC_ECUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return LSMC_OK;
}

}  // namespace

extern "C" int lsmc_backward_noalloc(const void* d_S, const void* d_V, uint32_t n_paths,
                                     uint32_t n_steps, int32_t precision,
                                     const lsmc_heston* model, const lsmc_contract* contract,
                                     int32_t basis, double* d_out, double* d_beta,
                                     uint32_t* d_n_singular, void* cuda_stream) {
  if (!d_S || !model || !contract || !d_out) return LSMC_EINVAL;
  void* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc) return rc;
  return lsmc::backward_in_scratch(scratch, kScratchBytes, d_S, d_V, n_paths, n_steps, precision,
                                   model, contract, basis, d_out, d_beta, d_n_singular,
                                   (cudaStream_t)cuda_stream);
}
