// FP32 throughput probe: the denominator of the ALU roofline, measured on the
// GPU the library runs on instead of derived from unit counts.
//
// Every thread runs 8 independent fma chains (enough independent work to hide
// the fma latency at full occupancy); the grid fills every SM at the kernel's
// maximum occupancy.  The scalar form issues one FP32 fma per lane and
// instruction; the paired form (fma.rn.f32x2) two.  The flop count is
// 2 per fma, the convention of the FP32 peak.
#include <cuda_runtime.h>

#include "hp_internal.h"

namespace hp {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeUnroll = 16;

__device__ float g_probe_sink;   // written only if a chain reached an impossible value

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, float a, float b) {
  float x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = 1e-3f * (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = __fmaf_rn(x[c], a, b);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  if (s == -1.0f) g_probe_sink = s;   // never true (the chains stay positive); keeps them live
}

__global__ void __launch_bounds__(kProbeThreads) k_fma2_probe(int iters, float a, float b) {
  unsigned long long x[4];
  const unsigned long long av = ((unsigned long long)__float_as_uint(a) << 32) | __float_as_uint(a);
  const unsigned long long bv = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float lo = 1e-3f * (float)(threadIdx.x + 2 * c), hi = 1e-3f * (float)(threadIdx.x + 2 * c + 1);
    x[c] = ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < 4; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += __uint_as_float((unsigned)x[c]) + __uint_as_float((unsigned)(x[c] >> 32));
  if (s == -1.0f) g_probe_sink = s;
}

}  // namespace
}  // namespace hp

extern "C" hp_status hp_measure_fp32_peak(int paired, int iters, int launches, void* stream, double* flops_per_s,
                                          double* ms_per_launch, int* sm_count) {
  using namespace hp;
  if (!flops_per_s || iters < 1 || launches < 1)
    return report_error(HP_ERR_INVALID_ARG, "hp_measure_fp32_peak: null result pointer or non-positive counts");
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  void (*kern)(int, float, float) = paired ? k_fma2_probe : k_fma_probe;
  if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kProbeThreads, 0);
  if (e || sms < 1 || per_sm < 1) {
    cudaGetLastError();
    return report_error(HP_ERR_CUDA, "hp_measure_fp32_peak: device query failed");
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = sms * per_sm;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaEventCreate(&ev[0]);
  if (!e) e = cudaEventCreate(&ev[1]);
  const float a = 0.9999999f, b = 1e-7f;
  if (!e) {
    kern<<<blocks, kProbeThreads, 0, s>>>(iters, a, b);   // warm-up
    e = cudaGetLastError();
  }
  if (!e) e = cudaEventRecord(ev[0], s);
  for (int i = 0; i < launches && !e; ++i) {
    kern<<<blocks, kProbeThreads, 0, s>>>(iters, a, b);
    e = cudaGetLastError();
    __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  }
  if (!e) e = cudaEventRecord(ev[1], s);
  if (!e) e = cudaEventSynchronize(ev[1]);
  float ms = 0.0f;
  if (!e) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  if (e) return report_error(HP_ERR_CUDA, cudaGetErrorString(e));
  const double fma_per_thread = (double)iters * kProbeUnroll * 8.0;   // 8 lanes of work either way
  const double flops = 2.0 * fma_per_thread * kProbeThreads * blocks * launches;
  *flops_per_s = flops / (ms * 1e-3);
  if (ms_per_launch) *ms_per_launch = ms / launches;
  if (sm_count) *sm_count = sms;
  return HP_OK;
}
