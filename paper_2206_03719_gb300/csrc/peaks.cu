// peaks.cu -- lsmc_measure_peaks: timed throughput of the arithmetic pipes the
// kernels of this library are bound by, the denominators of their roofline
// fractions: the FP64 fused multiply-add (the FP64 path), the FP32 fused
// multiply-add and the special-function unit (the single-precision stepper's
// square roots, reciprocals, logarithms and exponentials).  Each probe runs
// independent dependency chains on every thread of a grid that fills every
// SM, long enough (tens of milliseconds) for the clock to settle, timed with
// CUDA events, the fastest of five launches after two warm-up launches.
// Nothing about the device's settings is read or changed.
#include <cuda_runtime.h>

#include "../../include/lsmc.h"

namespace lsmc {
namespace {

constexpr int kChains = 8;       // independent chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

// where a probe would store its chains' sum if it ever equalled 1234.5 (it
// does not: the store keeps the chains from being optimised away)
static __device__ double g_sink[2];

// FP64: a <- a b + c on kChains chains; b just below 1 keeps the values bounded
__global__ void __launch_bounds__(kThreads) dfma_probe(int iters, double b) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 1.0 + 1e-3 * j + 1e-9 * threadIdx.x;
  const double c = 1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 1234.5) g_sink[0] = s;
}

__global__ void __launch_bounds__(kThreads) ffma_probe(int iters, float b) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 1.0f + 1e-3f * j + 1e-6f * threadIdx.x;
  const float c = 1e-4f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 1234.5f) g_sink[1] = s;
}

// special-function unit: a <- 2^(-a), which stays in (1/2, 1)
__device__ __forceinline__ float ex2_neg(float a) {
  float r;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-a));
  return r;
}

__global__ void __launch_bounds__(kThreads) xu_probe(int iters) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 0.5f + 0.01f * j + 1e-6f * threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = ex2_neg(a[j]);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 1234.5f) g_sink[1] = s;
}

// device milliseconds of the fastest of kReps launches (after two warm-up
// launches, so the clock has left its idle state)
constexpr int kReps = 5;
template <typename Launch>
cudaError_t time_ms(Launch launch, cudaStream_t s, float* ms) {
  cudaEvent_t ev[kReps + 1] = {};
  cudaError_t e = cudaSuccess;
  for (int i = 0; i <= kReps && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
  for (int i = 1; i <= kReps && e == cudaSuccess; ++i) {
    e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(ev[i], s);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[kReps]);
  float best = 0.0f;
  for (int i = 1; i <= kReps && e == cudaSuccess; ++i) {
    float t = 0.0f;
    e = cudaEventElapsedTime(&t, ev[i - 1], ev[i]);
    if (e == cudaSuccess && (i == 1 || t < best)) best = t;
  }
  for (int i = 0; i <= kReps; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  *ms = best;
  return e;
}

}  // namespace
}  // namespace lsmc

extern "C" int lsmc_measure_peaks(int32_t device, lsmc_peaks* out) {
  using namespace lsmc;
  if (!out) return LSMC_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) return LSMC_ENODEV;
  if (device < 0 || device >= ndev) return LSMC_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return LSMC_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = (sms > 0 ? sms : 1) * kBlocksPerSM;
  const double threads = (double)blocks * kThreads;
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  // iterations of 16 x kChains operations per thread: about 10 to 20 ms per
  // launch on a GB300
  const int it64 = 200, it32 = 16384, itxu = 4096;
  float ms[3] = {0.f, 0.f, 0.f};
  if (e == cudaSuccess)
    e = time_ms([&] {
      dfma_probe<<<blocks, kThreads, 0, s>>>(it64, 0.9999999);
      return cudaGetLastError();
    }, s, &ms[0]);
  if (e == cudaSuccess)
    e = time_ms([&] {
      ffma_probe<<<blocks, kThreads, 0, s>>>(it32, 0.9999f);
      return cudaGetLastError();
    }, s, &ms[1]);
  if (e == cudaSuccess)
    e = time_ms([&] {
      xu_probe<<<blocks, kThreads, 0, s>>>(itxu);
      return cudaGetLastError();
    }, s, &ms[2]);
  if (s) cudaStreamDestroy(s);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LSMC_ENOMEM : LSMC_ECUDA;
  const double ops = threads * 16.0 * kChains;  // operations per iteration of the grid
  out->fp64_tflops = 2.0 * ops * it64 / (ms[0] * 1e-3) / 1e12;
  out->fp32_tflops = 2.0 * ops * it32 / (ms[1] * 1e-3) / 1e12;
  out->xu_tops = ops * itxu / (ms[2] * 1e-3) / 1e12;
  out->fp64_ms = ms[0];
  out->fp32_ms = ms[1];
  out->xu_ms = ms[2];
  out->sms = sms;
  out->reserved = 0;
  return LSMC_OK;
}
