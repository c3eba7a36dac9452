// Learned right-eye reprojection: forward warp, network features, labels,
// retrace mask and composition (sm_103a).
//
// The paper computes both channels of a stereo pair independently (Sec. 3,
// "parallel level 1"). This extension renders the left channel, warps it to
// the right eye, and re-traces only the right pixels a small network (or a
// disocclusion hole) marks; the full right-eye trace remains the reference
// it is judged against.
//
// Forward warp (both eyes share the window on the convergence plane, so a
// left pixel at view depth z moves horizontally by the disparity
// D = f_px * s * (1/z - 1/zc) pixels, f_px = (H/2)/tan(vfov/2)):
//   x_R = i_L - D, target column i_R = floor(x_R + 0.5), same row. A z-test
//   keeps the nearest source: a 64-bit atomicMin of (z bits << 32 | left
//   index), so equal depths resolve to the lower left index. A left pixel
//   whose ray missed the scene is a source at infinity (z = +inf, D =
//   -f_px s / zc): it carries the background and loses every z-test, so only
//   true disocclusions and the uncovered image border stay holes.
// The disparity and the target column use explicitly rounded FP32
// operations (no contraction) so the decision is reproducible bit for bit.
//
// Features of a right pixel (10 channels, zeros on a hole):
//   min(z/100, 1), normal (3), hash(id) = (fmix32(id) >> 8) * 2^-24 with
//   MurmurHash3's 32-bit finaliser, left RGB (3), D/16, and the reflectivity
//   of the surface the left pixel hit: a mirror's colour depends on the
//   viewpoint, so warped mirror pixels are wrong however exact the warp, and
//   without this channel the network cannot see which pixels are mirrors.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_internal.cuh"

namespace rt {
namespace {

constexpr float kZFar = 100.f;
constexpr float kDispScale = 1.f / 16.f;
constexpr int kFeat = 10;          // feature channels (of the 16 stored per pixel)

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__device__ __forceinline__ float disparity(float z, float fs, float inv_zc) {
  return __fmul_rn(fs, __fsub_rn(__frcp_rn(z), inv_zc));
}

__global__ void k_warp_clear(unsigned long long* zbuf, uint32_t P) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x)
    zbuf[i] = ~0ull;
}

__global__ void k_warp_scatter(const float* __restrict__ depth_L, uint32_t W, uint32_t H, float fs,
                               float inv_zc, unsigned long long* zbuf) {
  const uint32_t P = W * H;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const float z = depth_L[p];
    if (!(z > 0.f)) continue;      // invalid depth; a miss (+inf) is a source at infinity
    const uint32_t j = p / W, i = p - j * W;
    const float xr = __fsub_rn((float)i, disparity(z, fs, inv_zc));
    const float c = floorf(__fadd_rn(xr, 0.5f));
    if (!(c >= 0.f) || !(c < (float)W)) continue;
    const unsigned long long key = ((unsigned long long)__float_as_uint(z) << 32) | p;
    atomicMin(zbuf + (size_t)j * W + (uint32_t)c, key);
  }
}

// features (bf16, 16 channels: 9 used + 7 zero pad; and optionally FP32 9
// channels), hole flags, warped RGB
__global__ void k_warp_gather(const unsigned long long* __restrict__ zbuf,
                              const float* __restrict__ depth_L, const float* __restrict__ normal_L,
                              const uint32_t* __restrict__ id_L, const float* __restrict__ rgb_L,
                              const float* __restrict__ refl_L, uint32_t P, float fs, float inv_zc,
                              __nv_bfloat16* feat16,
                              float* feat32, uint8_t* hole, float* warped) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const unsigned long long key = zbuf[p];
    float f[kFeat] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const bool h = key == ~0ull;
    if (!h) {
      const uint32_t q = (uint32_t)(key & 0xFFFFFFFFull);
      const float z = depth_L[q];
      f[0] = fminf(z * (1.f / kZFar), 1.f);
      f[1] = normal_L[3 * (size_t)q + 0];
      f[2] = normal_L[3 * (size_t)q + 1];
      f[3] = normal_L[3 * (size_t)q + 2];
      f[4] = (float)(fmix32(id_L[q]) >> 8) * 0x1p-24f;
      f[5] = rgb_L[3 * (size_t)q + 0];
      f[6] = rgb_L[3 * (size_t)q + 1];
      f[7] = rgb_L[3 * (size_t)q + 2];
      f[8] = disparity(z, fs, inv_zc) * kDispScale;
      f[9] = refl_L ? refl_L[q] : 0.f;
    }
    if (feat16) {                          // 32 bytes per pixel as two 16-byte stores
      uint32_t w[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float lo = 2 * c < kFeat ? f[2 * c] : 0.f, hi = 2 * c + 1 < kFeat ? f[2 * c + 1] : 0.f;
        __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        w[c] = *reinterpret_cast<uint32_t*>(&h);
      }
      uint4* o = reinterpret_cast<uint4*>(feat16 + 16 * (size_t)p);
      o[0] = make_uint4(w[0], w[1], w[2], w[3]);
      o[1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
    if (feat32) {
#pragma unroll
      for (int c = 0; c < kFeat; ++c) feat32[kFeat * (size_t)p + c] = f[c];
    }
    // 1: a hole; 2: the source surface reflects (its colour depends on the
    // viewpoint, so the warped colour is not the right eye's); the retrace
    // mask takes both, the training labels only the holes
    if (hole) hole[p] = h ? 1 : (f[9] > 0.f ? 2 : 0);
    if (warped) {
      warped[3 * (size_t)p + 0] = f[5];
      warped[3 * (size_t)p + 1] = f[6];
      warped[3 * (size_t)p + 2] = f[7];
    }
  }
}

// label = hole or max over channels |warped - full| > thr
__global__ void k_labels(const uint8_t* __restrict__ hole, const float* __restrict__ warped,
                         const float* __restrict__ full_R, uint32_t P, float thr, float* label) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    float e = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) e = fmaxf(e, fabsf(warped[3 * (size_t)p + c] - full_R[3 * (size_t)p + c]));
    label[p] = (hole[p] == 1 || e > thr) ? 1.f : 0.f;
  }
}

// mask = hole, reflective source, or prob > threshold; the masked right
// pixels (as global indices P + p) are appended to plist, in pixel order
// within each warp's 128 pixels, with one atomic per warp. A thread takes 4
// consecutive pixels (one 4-byte and one 16-byte load when the buffers allow
// it); the pixels past the last whole group of 4 are read one by one.
__global__ void k_mask_compact(const uint8_t* __restrict__ hole, const float* __restrict__ prob,
                               uint32_t P, float threshold, bool wide, uint8_t* mask,
                               uint32_t* plist, uint32_t* count) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t groups = (P + 3u) / 4u;
  for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < groups;
       base += gridDim.x * blockDim.x) {
    const uint32_t g = base + lane, p0 = 4u * g;
    uint32_t bits = 0;                    // bit j: pixel p0 + j is masked
    if (g < groups) {
      if (wide && p0 + 4u <= P) {
        const uchar4 h = *reinterpret_cast<const uchar4*>(hole + p0);
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (prob) q = *reinterpret_cast<const float4*>(prob + p0);
        bits = (h.x || (prob && q.x > threshold) ? 1u : 0u) | (h.y || (prob && q.y > threshold) ? 2u : 0u) |
               (h.z || (prob && q.z > threshold) ? 4u : 0u) | (h.w || (prob && q.w > threshold) ? 8u : 0u);
        if (mask)
          *reinterpret_cast<uchar4*>(mask + p0) =
              make_uchar4(bits & 1u, (bits >> 1) & 1u, (bits >> 2) & 1u, (bits >> 3) & 1u);
      } else {
        for (uint32_t j = 0; j < 4u && p0 + j < P; ++j) {
          const bool m = hole[p0 + j] || (prob && prob[p0 + j] > threshold);
          bits |= (m ? 1u : 0u) << j;
          if (mask) mask[p0 + j] = m ? 1 : 0;
        }
      }
    }
    // exclusive prefix sum of the lanes' counts
    const uint32_t n = __popc(bits);
    uint32_t incl = n;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if (lane >= (uint32_t)d) incl += v;
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    uint32_t off = 0;
    if (lane == 31 && total) off = atomicAdd(count, total);
    off = __shfl_sync(0xFFFFFFFFu, off, 31) + incl - n;
    for (uint32_t j = 0; j < 4u; ++j)
      if (bits >> j & 1u) plist[off++] = P + p0 + j;
  }
}

// right image: traced colour where masked, warped colour elsewhere
__global__ void k_compose(const uint8_t* __restrict__ mask, const uint32_t* __restrict__ accum_R,
                          const float* __restrict__ warped, uint32_t P, float inv_scale,
                          float* out_R) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < 3 * P; k += gridDim.x * blockDim.x) {
    const uint32_t p = k / 3;
    out_R[k] = mask[p] ? fminf(1.f, (float)accum_R[k] * inv_scale) : warped[k];
  }
}

// the same, 4 pixels (12 floats) per thread as 16-byte loads and stores;
// the sums are read only for groups with a masked pixel
__global__ void k_compose4(const uchar4* __restrict__ mask, const uint4* __restrict__ accum_R,
                           const float4* __restrict__ warped, uint32_t groups, float inv_scale,
                           float4* out_R) {
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += gridDim.x * blockDim.x) {
    const uchar4 m = mask[g];
    float4 v[3] = {warped[3 * (size_t)g], warped[3 * (size_t)g + 1], warped[3 * (size_t)g + 2]};
    if (m.x | m.y | m.z | m.w) {
      const uint4 a[3] = {accum_R[3 * (size_t)g], accum_R[3 * (size_t)g + 1], accum_R[3 * (size_t)g + 2]};
      const uint32_t* ai = reinterpret_cast<const uint32_t*>(a);
      float* vf = reinterpret_cast<float*>(v);
      const uint8_t mm[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (mm[j]) {
#pragma unroll
          for (int c = 0; c < 3; ++c) vf[3 * j + c] = fminf(1.f, (float)ai[3 * j + c] * inv_scale);
        }
    }
    out_R[3 * (size_t)g] = v[0];
    out_R[3 * (size_t)g + 1] = v[1];
    out_R[3 * (size_t)g + 2] = v[2];
  }
}

int grid_1d(uint64_t n, int threads) {
  uint64_t b = (n + threads - 1) / threads;
  const uint64_t cap = (uint64_t)num_sms() * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

cudaError_t reproj_warp(const float* depth_L, const float* normal_L, const uint32_t* id_L,
                        const float* rgb_L, const float* refl_L, uint32_t W, uint32_t H, float f_px, float eye_sep,
                        float convergence, unsigned long long* zbuf, __nv_bfloat16* feat16,
                        float* feat32, uint8_t* hole, float* warped, cudaStream_t st) {
  const uint32_t P = W * H;
  const float fs = f_px * eye_sep;
  const float inv_zc = 1.f / convergence;
  k_warp_clear<<<grid_1d(P, 256), 256, 0, st>>>(zbuf, P);
  k_warp_scatter<<<grid_1d(P, 256), 256, 0, st>>>(depth_L, W, H, fs, inv_zc, zbuf);
  k_warp_gather<<<grid_1d(P, 256), 256, 0, st>>>(zbuf, depth_L, normal_L, id_L, rgb_L, refl_L, P, fs,
                                                  inv_zc, feat16, feat32, hole, warped);
  return cudaGetLastError();
}

cudaError_t reproj_labels(const uint8_t* hole, const float* warped, const float* full_R, uint32_t P,
                          float thr, float* label, cudaStream_t st) {
  k_labels<<<grid_1d(P, 256), 256, 0, st>>>(hole, warped, full_R, P, thr, label);
  return cudaGetLastError();
}

cudaError_t reproj_mask(const uint8_t* hole, const float* prob, uint32_t P, float threshold,
                        uint8_t* mask, uint32_t* plist, uint32_t* count, cudaStream_t st) {
  cudaMemsetAsync(count, 0, sizeof(uint32_t), st);
  const bool wide = ((uintptr_t)hole % 4) == 0 && ((uintptr_t)prob % 16) == 0 && ((uintptr_t)mask % 4) == 0;
  k_mask_compact<<<grid_1d((P + 3) / 4, 256), 256, 0, st>>>(hole, prob, P, threshold, wide, mask, plist,
                                                            count);
  return cudaGetLastError();
}

cudaError_t reproj_compose(const uint8_t* mask, const uint32_t* accum_R, const float* warped,
                           uint32_t P, float inv_scale, float* out_R, cudaStream_t st) {
  const bool wide = P % 4 == 0 && ((uintptr_t)mask % 4) == 0 && ((uintptr_t)accum_R % 16) == 0 &&
                    ((uintptr_t)warped % 16) == 0 && ((uintptr_t)out_R % 16) == 0;
  if (wide)
    k_compose4<<<grid_1d(P / 4, 256), 256, 0, st>>>(reinterpret_cast<const uchar4*>(mask),
                                                    reinterpret_cast<const uint4*>(accum_R),
                                                    reinterpret_cast<const float4*>(warped), P / 4,
                                                    inv_scale, reinterpret_cast<float4*>(out_R));
  else
    k_compose<<<grid_1d(3ull * P, 256), 256, 0, st>>>(mask, accum_R, warped, P, inv_scale, out_R);
  return cudaGetLastError();
}

}  // namespace rt
