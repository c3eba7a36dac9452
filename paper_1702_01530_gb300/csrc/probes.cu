// Roofline probes (sm_103a): L2 read bandwidth and MUFU throughput.
//
// Neither ceiling is published for this part; the traversal's roofline uses
// them as a second bound (MUFU: one rcp per triangle test, one sqrt per
// sphere test, one rsqrt per normalised direction) and as a diagnostic (the
// bytes rays fetch from the L2-resident BVH).
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_internal.cuh"
#include "rt_probes.h"

namespace rt {
namespace {

constexpr int kL2Threads = 512, kL2PerSm = 4;
constexpr int kMufuThreads = 256, kMufuPerSm = 8;

__global__ void __launch_bounds__(kL2Threads) k_l2_read(const uint4* __restrict__ buf, uint64_t n,
                                                        uint32_t reps, uint4* __restrict__ sink) {
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  uint4 acc = make_uint4(0u, 0u, 0u, 0u);
  for (uint32_t r = 0; r < reps; ++r) {
    // rotate the start by a few CTAs' worth per pass; loads bypass L1 anyway
    const uint64_t shift = ((uint64_t)r * 7919u * blockDim.x) % n;
#pragma unroll 4
    for (uint64_t i = tid; i < n; i += nthreads) {
      uint64_t j = i + shift;
      if (j >= n) j -= n;
      const uint4 v = __ldcg(buf + j);
      acc.x ^= v.x; acc.y ^= v.y; acc.z ^= v.z; acc.w ^= v.w;
    }
  }
  sink[tid] = acc;
}

__global__ void __launch_bounds__(kMufuThreads) k_mufu(uint32_t iters, float* __restrict__ sink) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1.0f + (float)(threadIdx.x + 32 * k) * 1e-3f;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(x[k]));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  sink[blockIdx.x * (uint64_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace rt

extern "C" uint64_t rt_probe_l2_threads(void) {
  return (uint64_t)rt::num_sms() * rt::kL2PerSm * rt::kL2Threads;
}

extern "C" uint64_t rt_probe_mufu_threads(void) {
  return (uint64_t)rt::num_sms() * rt::kMufuPerSm * rt::kMufuThreads;
}

extern "C" int rt_probe_l2_read(const void* buf, uint64_t n_vec, uint32_t reps, void* sink,
                                uint64_t n_sink, void* cuda_stream) {
  if (!buf || !sink || n_vec == 0 || reps == 0 || ((uintptr_t)buf & 15u) || ((uintptr_t)sink & 15u))
    return rt::fail(RT_ERR_INVALID_ARG, "rt_probe_l2_read: bad argument");
  if (n_sink < rt_probe_l2_threads())
    return rt::fail(RT_ERR_INVALID_ARG, "rt_probe_l2_read: sink smaller than the grid");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  rt::k_l2_read<<<rt::num_sms() * rt::kL2PerSm, rt::kL2Threads, 0, st>>>(
      static_cast<const uint4*>(buf), n_vec, reps, static_cast<uint4*>(sink));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RT_OK : rt::cuda_fail(e, "rt_probe_l2_read");
}

extern "C" int rt_probe_mufu(uint32_t iters, float* sink, uint64_t n_sink, void* cuda_stream) {
  if (!sink || iters == 0) return rt::fail(RT_ERR_INVALID_ARG, "rt_probe_mufu: bad argument");
  if (n_sink < rt_probe_mufu_threads())
    return rt::fail(RT_ERR_INVALID_ARG, "rt_probe_mufu: sink smaller than the grid");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  rt::k_mufu<<<rt::num_sms() * rt::kMufuPerSm, rt::kMufuThreads, 0, st>>>(iters, sink);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RT_OK : rt::cuda_fail(e, "rt_probe_mufu");
}
