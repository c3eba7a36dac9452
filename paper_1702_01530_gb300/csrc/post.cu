// Stereo-pair post-processing for display (sm_103a).
//
// Paper Sec. 3: after the two channels are synthesised, GPU post-processing
// converts the stereo pair into the frame format of the display device, for
// example an anaglyph. Modes (FP32 RGB, row 0 at the top):
//   RT_COMPOSITE_ANAGLYPH_COLOR: (L.r, R.g, R.b)
//   RT_COMPOSITE_ANAGLYPH_GRAY:  (y(L), y(R), y(R)), y = 0.299 r + 0.587 g + 0.114 b
//                                evaluated as fma(0.114, b, fma(0.587, g, 0.299 r))
//   RT_COMPOSITE_SIDE_BY_SIDE:   an H x 2W image, left eye in the left half
// Memory-bound: 24 bytes read and 12 (24 side by side) written per pixel,
// float4-wide where the row layout allows.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_internal.cuh"

namespace rt {
namespace {

__device__ __forceinline__ float luma(float r, float g, float b) {
  return fmaf(0.114f, b, fmaf(0.587f, g, 0.299f * r));
}

__global__ void k_anaglyph(const float* __restrict__ L, const float* __restrict__ R, uint32_t P,
                           int gray, float* __restrict__ out) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const float lr = L[3 * (size_t)p], lg = L[3 * (size_t)p + 1], lb = L[3 * (size_t)p + 2];
    const float rr = R[3 * (size_t)p], rg = R[3 * (size_t)p + 1], rb = R[3 * (size_t)p + 2];
    float o0, o1, o2;
    if (gray) {
      o0 = luma(lr, lg, lb);
      o1 = o2 = luma(rr, rg, rb);
    } else {
      o0 = lr; o1 = rg; o2 = rb;
    }
    out[3 * (size_t)p] = o0;
    out[3 * (size_t)p + 1] = o1;
    out[3 * (size_t)p + 2] = o2;
  }
}

// side by side: output row j = [L row j | R row j], copied as float4 when
// the row length (3W floats) is a multiple of 4
__global__ void k_side_by_side(const float* __restrict__ L, const float* __restrict__ R, uint32_t W,
                               uint32_t H, float* __restrict__ out) {
  const uint32_t row = 3 * W;
  if ((row & 3u) == 0 && (((uintptr_t)L | (uintptr_t)R | (uintptr_t)out) & 15u) == 0) {
    const uint32_t q = row / 4;                // float4 per eye row
    const uint64_t n = (uint64_t)2 * q * H;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
      const uint64_t j = i / (2 * q), c = i - j * 2 * q;
      const float4* src = reinterpret_cast<const float4*>(c < q ? L : R) + j * q + (c < q ? c : c - q);
      reinterpret_cast<float4*>(out)[i] = *src;
    }
    return;
  }
  const uint64_t n = (uint64_t)2 * row * H;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t j = i / (2 * row), c = i - j * 2 * row;
    out[i] = c < row ? L[j * row + c] : R[j * row + c - row];
  }
}

}  // namespace
}  // namespace rt

extern "C" int rt_stereo_composite(const float* d_L, const float* d_R, uint32_t W, uint32_t H,
                                   int mode, float* d_out, void* cuda_stream) {
  if (!d_L || !d_R || !d_out || W < 1 || H < 1 || (uint64_t)W * H > (1ull << 31) || mode < 0 || mode > 2)
    return rt::fail(RT_ERR_INVALID_ARG, "bad argument");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int grid = rt::num_sms() * 8;
  if (mode == RT_COMPOSITE_SIDE_BY_SIDE)
    rt::k_side_by_side<<<grid, 256, 0, st>>>(d_L, d_R, W, H, d_out);
  else
    rt::k_anaglyph<<<grid, 256, 0, st>>>(d_L, d_R, W * H, mode == RT_COMPOSITE_ANAGLYPH_GRAY, d_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rt::cuda_fail(e, "composite");
  return RT_OK;
}
