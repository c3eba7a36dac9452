// rt_build_lbvh_noalloc: the linear-BVH build for callers that cannot
// allocate device memory.
//
// rt_scene_create allocates its own buffers with cudaMalloc. Some callers
// cannot do that: code embedded in a host application that hands out all
// device memory through its own pool and forbids raw cudaMalloc, or a
// real-time loop that must not pay for cudaMalloc's implicit device
// synchronisation in the middle of a frame. This entry point runs the same
// build kernels as rt_scene_create (lbvh.cu) into buffers the caller owns,
// and keeps its scratch in one file-scope __device__ array, so it performs
// no allocation of any kind.
//
// The array is kNoAllocScratchBytes (13 MiB) on every GPU that loads this
// library, held until the process exits; it bounds a build to
// kNoAllocMaxPrims primitives. Every call shares the array, so calls whose
// GPU work overlaps (different streams, or different host threads) race on
// it; calls issued one after another on one stream are fine. Whatever must
// start at zero (the refit arrival counters, the error word) is cleared by
// each call.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "rt_internal.cuh"

namespace {

constexpr uint32_t kNoAllocMaxPrims = 1u << 20;
constexpr size_t kNoAllocScratchBytes = 13u << 20;
constexpr size_t kErrOffset = kNoAllocScratchBytes - 256;  // error word at the end

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

int fail(int code, const std::string& msg) {
  rt_set_error(msg);
  return code;
}

// Device address of the scratch array in the current context. The host-side
// symbol is not a device address, and the device address belongs to the
// context that loaded the module (a device reset or another context on the
// same device loads it again, possibly elsewhere), so it is looked up on
// every call; the lookup is cheap next to a build that synchronises.
int scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return fail(RT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  *out = p;
  return RT_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" int rt_build_lbvh_noalloc(const rt_sphere* d_spheres, uint32_t n_spheres,
                                     const rt_triangle* d_tris, uint32_t n_tris, float* d_nodes,
                                     float* d_prims, uint64_t* d_keys, int32_t* d_parent,
                                     void* cuda_stream) {
  const uint64_t n = (uint64_t)n_spheres + n_tris;
  if (n < 1) return fail(RT_ERR_INVALID_ARG, "need at least one primitive");
  if (n > kNoAllocMaxPrims)
    return fail(RT_ERR_INVALID_ARG, "rt_build_lbvh_noalloc: " + std::to_string(n) +
                                        " primitives exceed its limit of " +
                                        std::to_string(kNoAllocMaxPrims) +
                                        " (use rt_scene_create for larger scenes)");
  if ((n_spheres && !d_spheres) || (n_tris && !d_tris) || !d_nodes || !d_prims || !d_keys || !d_parent)
    return fail(RT_ERR_INVALID_ARG, "a required device pointer is NULL");
  if (!aligned16(d_nodes) || !aligned16(d_prims))
    return fail(RT_ERR_INVALID_ARG, "d_nodes and d_prims must be 16-byte aligned");
  const size_t need = rt::lbvh_tmp_bytes((uint32_t)n);
  if (need > kErrOffset) return fail(RT_ERR_INVALID_ARG, "scratch too small for this build");
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  uint32_t* d_err = reinterpret_cast<uint32_t*>(static_cast<char*>(base) + kErrOffset);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess)
    e = rt::build_lbvh(reinterpret_cast<const float4*>(d_spheres), reinterpret_cast<const float*>(d_tris),
                       n_spheres, n_tris, reinterpret_cast<float4*>(d_nodes),
                       reinterpret_cast<float4*>(d_prims), d_keys, d_parent, base, kErrOffset, d_err, st);
  uint32_t bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, d_err, sizeof bits, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(RT_ERR_CUDA, std::string("rt_build_lbvh_noalloc: ") + cudaGetErrorString(e));
  if (bits) return fail(RT_ERR_DEVICE_CHECK, "BVH build device check failed (bits " + std::to_string(bits) + ")");
  return RT_OK;
}
