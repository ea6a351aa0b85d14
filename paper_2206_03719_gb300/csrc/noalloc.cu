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
#include <cuda.h>  // driver types of the context query (no link to the driver library)
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lsmc.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB per device

// Every device that loads this library holds this array until the process
// exits.  In host code the name is only a host-side stand-in: its device
// address comes from cudaGetSymbolAddress, looked up per device and context.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// The address cudaGetSymbolAddress returns belongs to one CUDA context: the
// device's primary context is rebuilt after cudaDeviceReset, and a caller may
// run under a context of its own.  The cache is therefore keyed by the
// identity of the current context (cuCtxGetId, reached through the runtime's
// driver entry points so the library does not link the driver library).
using CtxGetCurrent = CUresult (*)(CUcontext*);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long*);

struct DriverQueries {
  CtxGetCurrent get_current = nullptr;
  CtxGetId get_id = nullptr;
};

const DriverQueries& driver_queries() {
  static const DriverQueries q = [] {
    DriverQueries d;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult st{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &st) ==
            cudaSuccess && st == cudaDriverEntryPointSuccess)
      d.get_current = reinterpret_cast<CtxGetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &st) ==
            cudaSuccess && st == cudaDriverEntryPointSuccess)
      d.get_id = reinterpret_cast<CtxGetId>(f);
    return d;
  }();
  return q;
}

// Identity of the calling thread's current context; false when it cannot be
// read or no context is current yet.
bool current_context_id(unsigned long long* id) {
  const DriverQueries& q = driver_queries();
  if (!q.get_current || !q.get_id) return false;
  CUcontext c = nullptr;
  if (q.get_current(&c) != CUDA_SUCCESS || !c) return false;
  return q.get_id(c, id) == CUDA_SUCCESS;
}

constexpr int kMaxDevices = 64;
struct CachedAddress {
  void* addr = nullptr;
  unsigned long long ctx_id = 0;
};
std::mutex g_mu;
CachedAddress g_addr[kMaxDevices];

// Device address of g_scratch in the current context of the current device:
// looked up on the first call of a (device, context) pair, then cached.  When
// the context cannot be identified the lookup runs on every call.
int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LSMC_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return LSMC_ENODEV;
  unsigned long long id = 0;
  bool keyed = current_context_id(&id);
  std::lock_guard<std::mutex> g(g_mu);
  CachedAddress& c = g_addr[dev];
  if (keyed && c.addr && c.ctx_id == id) {
    *out = c.addr;
    return LSMC_OK;
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return LSMC_ECUDA;
  // the lookup makes the device's primary context current if none was
  if (!keyed) keyed = current_context_id(&id);
  c.addr = keyed ? p : nullptr;
  c.ctx_id = id;
  *out = p;
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
