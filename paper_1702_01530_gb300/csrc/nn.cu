// Retrace-probability network: 4 layers of 3x3 convolutions
// (9 -> 32 -> 32 -> 32 -> 1, zero padding 1, ReLU, sigmoid), BF16 operands
// and FP32 accumulation on the 5th-generation tensor cores (sm_103a).
//
// Convolution as implicit GEMM on tcgen05:
//   a persistent CTA (128 threads) computes tiles of R rows x 128 consecutive
//   pixels: per row, D[128 pixels, Cout] = sum over the 9 taps (dy, dx) of
//   A_tap[128, Cin] x B_tap[Cin, Cout]. The input halo (R+2 rows x 130 pixels x
//   Cin channels, BF16) sits in shared memory as 16-byte (8-channel) chunks
//   ordered [chunk][halo pixel], so A_tap for every tap is the same matrix
//   shifted by (row+dy)*130 + dx rows: the K-major, non-swizzled operand layout
//   with 8-row core matrices 128 B apart (SBO) and 8-channel chunks
//   (R+2)*130*16 B apart (LBO). Weights are pre-packed in the same core-matrix
//   layout. Halos stream in with 16-byte cp.async copies (zero-filled
//   outside the image); with one buffer the next tile's copies start as soon
//   as the MMAs of this tile have consumed it, under the epilogue. One elected thread issues 9 * Cin/16 tcgen05.mma (M=128,
//   N=Cout, K=16, kind::f16 with BF16 inputs) into a TMEM accumulator,
//   commits to an mbarrier; the four warps read their 32 TMEM lanes
//   (tcgen05.ld 32x32b) for the fused epilogue (bias + ReLU -> BF16, or
//   bias + sigmoid -> FP32, or the backward ReLU mask).
//   Every mbarrier wait has an iteration bound; on expiry the kernel sets the
//   error word, skips the tile and still frees its TMEM.
//
// Backward pass: data gradients are convolutions with the 3x3 taps flipped
// and Cin/Cout swapped (same tensor-core kernel); weight gradients are an
// FP32 CUDA-core reduction over pixels; BCE on the sigmoid output; Adam on
// FP32 master weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdlib>

#include "rt_internal.cuh"

namespace rt {
namespace nn {

// Tuning knobs: RT_CONV_ROWS = image rows per tile (R accumulators of
// 128 pixels share one halo of R+2 rows); RT_CONV_DBUF = 1 double-buffers
// the halo (the next tile loads while this one computes). Measured on GB300
// at 1920x1080 (network forward, 4 layers, identical output bit for bit):
// R=1 0.52 ms, R=2 0.45-0.48, R=4 0.42-0.43, R=8 single-buffered 0.40 ms.
#ifndef RT_CONV_ROWS
#define RT_CONV_ROWS 8
#endif
#ifndef RT_CONV_DBUF
#define RT_CONV_DBUF 0
#endif
constexpr int kRows = RT_CONV_ROWS;
constexpr int kBufs = RT_CONV_DBUF ? 2 : 1;
constexpr int kTileM = 128;          // pixels per row tile (one MMA M block)
constexpr int kHaloW = kTileM + 2;   // 130
constexpr int kHaloRows = (kRows + 2) * kHaloW;  // halo pixels per tile
constexpr uint32_t kWaitBound = 1u << 26;

enum Epi : int { EPI_RELU_BF16 = 0, EPI_SIGMOID_F32 = 1, EPI_BWD_MASK_BF16 = 2 };

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory matrix descriptor, no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;  // descriptor version for tcgen05
  return d;        // base offset 0, relative LBO mode, swizzle none
}

// instruction descriptor: kind::f16, D = F32, A = B = BF16, both K-major
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < kWaitBound; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16-byte asynchronous global->shared copy; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// 16 consecutive TMEM columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// ------------------------------------------------------------ conv kernel
// in:  BF16 [P][CIN] activations (CIN = 16 or 32)
// wpk: BF16 packed weights, [tap][CIN/8][COUT][8]
// EPI_RELU_BF16:     out16[P][COUT] = relu(acc + bias)
// EPI_SIGMOID_F32:   out32[P] = sigmoid(acc[0] + bias[0])
// EPI_BWD_MASK_BF16: out16[P][COUT] = acc * (mask16[P][COUT] > 0)
template <int CIN>
__device__ __forceinline__ void load_halo_async(unsigned char* halo, const __nv_bfloat16* in,
                                                uint32_t tile, uint32_t tiles_x, uint32_t W,
                                                uint32_t H, int tid) {
  constexpr int kChunks = CIN / 8;
  const int ty = (int)(tile / tiles_x);
  const int y = ty * kRows;
  const int x0 = (int)(tile - (uint32_t)ty * tiles_x) * kTileM;
  // 16-byte chunk c of halo pixel r goes to ((c * kHaloRows) + r) * 16; consecutive
  // threads take consecutive halo pixels of one chunk (conflict-free stores)
  for (int k = tid; k < kHaloRows * kChunks; k += 128) {
    const int c = k / kHaloRows, r = k - c * kHaloRows;
    const int dy = r / kHaloW, xx = r - dy * kHaloW;
    const int gy = y + dy - 1, gx = x0 + xx - 1;
    const bool ok = gy >= 0 && gy < (int)H && gx >= 0 && gx < (int)W;
    const __nv_bfloat16* src = ok ? in + ((size_t)gy * W + gx) * CIN + c * 8 : in;
    cp_async16(halo + ((size_t)c * kHaloRows + r) * 16, src, ok ? 16u : 0u);
  }
}

template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(128) k_conv_tc(const __nv_bfloat16* __restrict__ in,
                                                  const __nv_bfloat16* __restrict__ wpk,
                                                  const float* __restrict__ bias,
                                                  const __nv_bfloat16* __restrict__ mask16,
                                                  __nv_bfloat16* __restrict__ out16,
                                                  float* __restrict__ out32, uint32_t W, uint32_t H,
                                                  uint32_t* err) {
  static_assert(CIN % 16 == 0 && (COUT == 16 || COUT == 32), "shape");
  constexpr int kChunks = CIN / 8;
  constexpr uint32_t kHaloBytes = kHaloRows * CIN * 2;
  constexpr uint32_t kHaloStride = (kHaloBytes + 1023) & ~1023u;
  constexpr uint32_t kWBytes = 9 * COUT * CIN * 2;
  constexpr uint32_t kLBO_A = kHaloRows * 16;   // next 8-channel chunk of the halo
  constexpr uint32_t kLBO_B = COUT * 16;        // next 8-channel chunk of a weight tap
  constexpr uint32_t kAccCols = kRows * COUT;   // one accumulator per output row
  constexpr uint32_t kTmemCols = kAccCols <= 32 ? 32 : (kAccCols <= 64 ? 64 : (kAccCols <= 128 ? 128 : 256));
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* halo0 = smem;                  // kBufs halo buffers
  unsigned char* wsm = smem + kBufs * kHaloStride;
  float* bsm = reinterpret_cast<float*>(wsm + ((kWBytes + 127) & ~127u));
  uint64_t* bar = reinterpret_cast<uint64_t*>(bsm + 32);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t tiles_x = (W + kTileM - 1) / kTileM;
  const uint32_t n_tiles = tiles_x * ((H + kRows - 1) / kRows);
  // first halo in flight while the weights are copied
  if (blockIdx.x < n_tiles) load_halo_async<CIN>(halo0, in, blockIdx.x, tiles_x, W, H, tid);
  cp_async_commit();
  {
    const uint4* src = reinterpret_cast<const uint4*>(wpk);
    uint4* dst = reinterpret_cast<uint4*>(wsm);
    for (uint32_t i = tid; i < kWBytes / 16; i += 128) dst[i] = src[i];
    if (tid < COUT) bsm[tid] = bias ? bias[tid] : 0.f;
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tslot, kTmemCols);
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = make_idesc(kTileM, COUT);
  uint32_t phase = 0;
  uint32_t it = 0;

  for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
    unsigned char* halo = halo0 + (kBufs == 2 ? (it & 1u) : 0u) * kHaloStride;
    const uint32_t next = tile + gridDim.x;
    if (kBufs == 2) {
      // next tile's halo into the other buffer (freed at the end of the last iteration)
      if (next < n_tiles)
        load_halo_async<CIN>(halo0 + ((it + 1) & 1u) * kHaloStride, in, next, tiles_x, W, H, tid);
      cp_async_commit();
      cp_async_wait_1();          // this tile's halo has landed
    } else {
      asm volatile("cp.async.wait_all;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const int ty = (int)(tile / tiles_x);
    const int y = ty * kRows;
    const int x0 = (int)(tile - (uint32_t)ty * tiles_x) * kTileM;
    if (tid == 0) {
      const uint32_t hbase = smem_u32(halo), wbase = smem_u32(wsm);
#pragma unroll
      for (int ry = 0; ry < kRows; ++ry) {
        uint32_t acc = 0;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const int dy = tap / 3, dx = tap % 3;
#pragma unroll
          for (int ks = 0; ks < CIN / 16; ++ks) {
            const uint64_t da = make_desc(
                hbase + (uint32_t)((2 * ks) * kHaloRows + (ry + dy) * kHaloW + dx) * 16u, kLBO_A, 128u);
            const uint64_t db =
                make_desc(wbase + (uint32_t)((tap * kChunks + 2 * ks) * COUT) * 16u, kLBO_B, 128u);
            mma_bf16(tmem + (uint32_t)(ry * COUT), da, db, idesc, acc);
            acc = 1;
          }
        }
      }
      mma_commit(bar);
    }
    const bool ok = mbar_wait(bar, phase);
    phase ^= 1u;
    fence_after();
    if (!ok) {
      if (tid == 0) atomicOr(err, ERR_ITER);
      break;                       // uniform: every thread saw the same barrier state
    }
    // epilogue: warp w owns TMEM lanes (pixels) 32w .. 32w + 31 of every row
    if (kBufs == 1 && next < n_tiles) {
      // single buffer: the halo was consumed by the MMAs (barrier passed), so
      // the next tile's loads may start under the epilogue
      fence_before();
      __syncthreads();
      fence_after();
      load_halo_async<CIN>(halo0, in, next, tiles_x, W, H, tid);
      cp_async_commit();
    }
    const int x = x0 + warp * 32 + lane;
#pragma unroll
    for (int ry = 0; ry < kRows; ++ry) {
      const int yy = y + ry;
      const bool valid = x < (int)W && yy < (int)H;
      const size_t p = (size_t)yy * W + x;
      const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ry * COUT);
      if (EPI == EPI_SIGMOID_F32) {
        float v[16];
        tmem_ld16(lane_addr, v);
        if (valid) out32[p] = 1.f / (1.f + __expf(-(v[0] + bsm[0])));
      } else {
#pragma unroll
        for (int half = 0; half < COUT / 16; ++half) {
          float v[16];
          tmem_ld16(lane_addr + half * 16, v);
          if (valid) {
            uint32_t packed[8];
            if (EPI == EPI_RELU_BF16) {
#pragma unroll
              for (int i = 0; i < 8; ++i)
                packed[i] = pack_bf16(fmaxf(v[2 * i] + bsm[half * 16 + 2 * i], 0.f),
                                      fmaxf(v[2 * i + 1] + bsm[half * 16 + 2 * i + 1], 0.f));
            } else {
              const uint4* m4 = reinterpret_cast<const uint4*>(mask16 + p * COUT + half * 16);
              const uint4 ma = m4[0], mb = m4[1];
              const uint32_t mw[8] = {ma.x, ma.y, ma.z, ma.w, mb.x, mb.y, mb.z, mb.w};
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const __nv_bfloat162 mm = *reinterpret_cast<const __nv_bfloat162*>(&mw[i]);
                const float m0 = __bfloat162float(mm.x), m1 = __bfloat162float(mm.y);
                packed[i] = pack_bf16(m0 > 0.f ? v[2 * i] : 0.f, m1 > 0.f ? v[2 * i + 1] : 0.f);
              }
            }
            uint4* o = reinterpret_cast<uint4*>(out16 + p * COUT + half * 16);
            o[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
            o[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
          }
        }
      }
    }
    fence_before();
    __syncthreads();  // TMEM read and this halo consumed before they are reused
    fence_after();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

template <int CIN, int COUT>
constexpr size_t conv_smem_bytes() {
  return kBufs * ((kHaloRows * CIN * 2 + 1023) & ~1023) + ((9 * COUT * CIN * 2 + 127) & ~127) + 32 * 4 + 16;
}

// ------------------------------------------------ weight packing (FP32 -> BF16)
// Canonical parameter layout of a layer: W[Cout][Cin][3][3] then b[Cout].
// forward pack: [tap][ci/8][co][ci%8] with ci < cin_pad, co < cout_pad (zero fill)
__global__ void k_pack_fwd(const float* __restrict__ Wt, int cout, int cin, int cout_pad,
                           int cin_pad, __nv_bfloat16* __restrict__ out) {
  const int n = 9 * cin_pad * cout_pad;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int e = i % 8, rest = i / 8;
    const int co = rest % cout_pad, rest2 = rest / cout_pad;
    const int chunk = rest2 % (cin_pad / 8), tap = rest2 / (cin_pad / 8);
    const int ci = chunk * 8 + e;
    float v = 0.f;
    if (co < cout && ci < cin) v = Wt[((size_t)co * cin + ci) * 9 + tap];
    out[i] = __float2bfloat16_rn(v);
  }
}

// backward-data pack: output channel = forward ci, input channel = forward co,
// tap flipped: W'[ci][co][8 - tap]
__global__ void k_pack_bwd(const float* __restrict__ Wt, int cout, int cin, int cout_pad,
                           int cin_pad, __nv_bfloat16* __restrict__ out) {
  // as a conv: CIN' = cout_pad, COUT' = cin_pad
  const int n = 9 * cout_pad * cin_pad;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int e = i % 8, rest = i / 8;
    const int ci = rest % cin_pad, rest2 = rest / cin_pad;      // output channel of the bwd conv
    const int chunk = rest2 % (cout_pad / 8), tap = rest2 / (cout_pad / 8);
    const int co = chunk * 8 + e;                               // input channel of the bwd conv
    float v = 0.f;
    if (co < cout && ci < cin) v = Wt[((size_t)co * cin + ci) * 9 + (8 - tap)];
    out[i] = __float2bfloat16_rn(v);
  }
}

// ------------------------------------------------------- BCE + d(logit)
// loss = mean(-(y log p + (1-y) log(1-p))), dlogit = p - y (the 1/P factor is
// applied in the weight-gradient kernel); dlogit goes to channel 0 of a
// 16-channel BF16 map (the input of the layer-4 data-gradient conv) and to an
// FP32 copy
__global__ void k_bce(const float* __restrict__ prob, const float* __restrict__ label, uint32_t P,
                      __nv_bfloat16* __restrict__ g16, float* __restrict__ g32,
                      float* __restrict__ loss_sum) {
  float acc = 0.f;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const float q = fminf(fmaxf(prob[p], 1e-7f), 1.f - 1e-7f), y = label[p];
    acc += -(y * __logf(q) + (1.f - y) * __logf(1.f - q));
    const float g = prob[p] - y;
    g32[p] = g;
    __nv_bfloat16* o = g16 + 16 * (size_t)p;
    o[0] = __float2bfloat16_rn(g);
#pragma unroll
    for (int c = 1; c < 16; ++c) o[c] = __float2bfloat16_rn(0.f);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss_sum, acc);
}

// ------------------------------------------------------ weight gradients
// dW[co][ci][ky][kx] += scale * sum_x dZ[y][x][co] * A[y+ky-1][x+kx-1][ci],
// db[co] += scale * sum_x dZ[y][x][co]; one CTA per image row, a 128-pixel
// chunk at a time through shared memory, FP32 accumulation, atomics at the end.
// dZ comes as FP32 (layer 4, one channel) or BF16 [P][dz_stride].
template <int CIN_PAD, int COUT>
__global__ void __launch_bounds__(256) k_wgrad(const __nv_bfloat16* __restrict__ A, int cin,
                                               const __nv_bfloat16* __restrict__ dz16,
                                               const float* __restrict__ dz32, int dz_stride,
                                               uint32_t W, uint32_t H, float scale,
                                               float* __restrict__ dW, float* __restrict__ db) {
  constexpr int kChunk = 64;
  constexpr int kOut = COUT * CIN_PAD * 9;
  constexpr int kPer = (kOut + 255) / 256;
  __shared__ float sA[3][kChunk + 2][CIN_PAD];
  __shared__ float sZ[kChunk][COUT];
  float acc[kPer];
  float bacc = 0.f;
#pragma unroll
  for (int i = 0; i < kPer; ++i) acc[i] = 0.f;
  const int tid = threadIdx.x;
  for (uint32_t y = blockIdx.x; y < H; y += gridDim.x) {
    for (uint32_t x0 = 0; x0 < W; x0 += kChunk) {
      __syncthreads();
      for (int k = tid; k < 3 * (kChunk + 2) * CIN_PAD; k += 256) {
        const int c = k % CIN_PAD, r = k / CIN_PAD;
        const int dy = r / (kChunk + 2), xx = r % (kChunk + 2);
        const int gy = (int)y + dy - 1, gx = (int)x0 + xx - 1;
        float v = 0.f;
        if (c < cin && gy >= 0 && gy < (int)H && gx >= 0 && gx < (int)W)
          v = __bfloat162float(A[((size_t)gy * W + gx) * CIN_PAD + c]);
        sA[dy][xx][c] = v;
      }
      for (int k = tid; k < kChunk * COUT; k += 256) {
        const int co = k % COUT, xx = k / COUT;
        const uint32_t gx = x0 + xx;
        float v = 0.f;
        if (gx < W) {
          const size_t p = (size_t)y * W + gx;
          v = dz32 ? dz32[p] : __bfloat162float(dz16[p * dz_stride + co]);
        }
        sZ[xx][co] = v;
      }
      __syncthreads();
      const int nx = (int)(W - x0 < (uint32_t)kChunk ? W - x0 : (uint32_t)kChunk);
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int o = tid + i * 256;
        if (o < kOut) {
          const int tap = o % 9, rest = o / 9;
          const int ci = rest % CIN_PAD, co = rest / CIN_PAD;
          const int dy = tap / 3, dx = tap % 3;
          float s = 0.f;
          for (int xx = 0; xx < nx; ++xx) s = fmaf(sZ[xx][co], sA[dy][xx + dx][ci], s);
          acc[i] += s;
        }
      }
      if (tid < COUT)
        for (int xx = 0; xx < nx; ++xx) bacc += sZ[xx][tid];
    }
  }
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int o = tid + i * 256;
    if (o < kOut) {
      const int tap = o % 9, rest = o / 9;
      const int ci = rest % CIN_PAD, co = rest / CIN_PAD;
      if (ci < cin) atomicAdd(&dW[((size_t)co * cin + ci) * 9 + tap], acc[i] * scale);
    }
  }
  if (tid < COUT) atomicAdd(&db[tid], bacc * scale);
}

// ---------------------------------------------------------------- Adam
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, uint32_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace nn
}  // namespace rt

// ===================================================================== host
namespace rt {
namespace nn {

namespace {
// extra dynamic shared memory per conv CTA (bytes), from RT_CONV_SMEM_PAD:
// lets a first run on new hardware keep every descriptor-addressed byte
// inside the CTA's allocation even under another reading of the layout
int conv_smem_pad() {
  static int pad = -1;
  if (pad < 0) {
    const char* v = getenv("RT_CONV_SMEM_PAD");
    pad = v ? atoi(v) : 0;
    if (pad < 0 || pad > 160 * 1024) pad = 0;
  }
  return pad;
}
int g_conv_smem_pad = 0;

template <int CIN, int COUT, int EPI>
cudaError_t launch_conv(const __nv_bfloat16* in, const __nv_bfloat16* wpk, const float* bias,
                        const __nv_bfloat16* mask16, __nv_bfloat16* out16, float* out32,
                        uint32_t W, uint32_t H, uint32_t* err, cudaStream_t st) {
  const size_t smem = conv_smem_bytes<CIN, COUT>() + (size_t)(g_conv_smem_pad + conv_smem_pad());
  static size_t configured = 0;
  if (configured < smem) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc<CIN, COUT, EPI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  // resident CTAs per SM from the shared-memory footprint (227 KB usable, 1 KB
  // reserved per CTA) and the TMEM columns each CTA allocates
  int per_sm = (int)((227u * 1024u) / (smem + 1024u));
  constexpr int kAcc = kRows * COUT;        // TMEM columns a CTA allocates (power of two >= 32)
  constexpr int kCols = kAcc <= 32 ? 32 : (kAcc <= 64 ? 64 : (kAcc <= 128 ? 128 : 256));
  if (per_sm > 512 / kCols) per_sm = 512 / kCols;   // 512 TMEM columns per SM
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 8) per_sm = 8;
  const uint32_t tiles = ((W + kTileM - 1) / kTileM) * ((H + kRows - 1) / kRows);
  uint32_t grid = (uint32_t)(num_sms() * per_sm);
  if (grid > tiles) grid = tiles;
  k_conv_tc<CIN, COUT, EPI><<<grid, 128, smem, st>>>(in, wpk, bias, mask16, out16, out32, W, H, err);
  return cudaGetLastError();
}
}  // namespace

void set_conv_smem_pad(int bytes) { g_conv_smem_pad = bytes; }

// parameter offsets (canonical layout W[Cout][Cin][3][3], b[Cout] per layer)
constexpr uint32_t kOffW[4] = {0, 2624, 11872, 21120};
constexpr uint32_t kOffB[4] = {2592, 11840, 21088, 21408};
constexpr int kCout[4] = {32, 32, 32, 1};
constexpr int kCin[4] = {9, 32, 32, 32};
constexpr int kCinPad[4] = {16, 32, 32, 32};
constexpr int kCoutPad[4] = {32, 32, 32, 16};

size_t packed_fwd_elems(int l) { return 9ull * kCinPad[l] * kCoutPad[l]; }
size_t packed_bwd_elems(int l) { return 9ull * kCoutPad[l] * kCinPad[l]; }

cudaError_t pack_weights(const float* params, __nv_bfloat16* const wf[4], __nv_bfloat16* const wb[4],
                         cudaStream_t st) {
  for (int l = 0; l < 4; ++l) {
    k_pack_fwd<<<64, 256, 0, st>>>(params + kOffW[l], kCout[l], kCin[l], kCoutPad[l], kCinPad[l], wf[l]);
    if (l > 0 && wb[l])
      k_pack_bwd<<<64, 256, 0, st>>>(params + kOffW[l], kCout[l], kCin[l], kCoutPad[l], kCinPad[l], wb[l]);
  }
  return cudaGetLastError();
}

cudaError_t forward(const __nv_bfloat16* feat16, const float* params, __nv_bfloat16* const wf[4],
                    __nv_bfloat16* act1, __nv_bfloat16* act2, __nv_bfloat16* act3, float* prob,
                    uint32_t W, uint32_t H, uint32_t* err, cudaStream_t st) {
  cudaError_t e;
  e = launch_conv<16, 32, EPI_RELU_BF16>(feat16, wf[0], params + kOffB[0], nullptr, act1, nullptr, W, H, err, st);
  if (e != cudaSuccess) return e;
  e = launch_conv<32, 32, EPI_RELU_BF16>(act1, wf[1], params + kOffB[1], nullptr, act2, nullptr, W, H, err, st);
  if (e != cudaSuccess) return e;
  e = launch_conv<32, 32, EPI_RELU_BF16>(act2, wf[2], params + kOffB[2], nullptr, act3, nullptr, W, H, err, st);
  if (e != cudaSuccess) return e;
  return launch_conv<32, 16, EPI_SIGMOID_F32>(act3, wf[3], params + kOffB[3], nullptr, nullptr, prob, W, H, err, st);
}

// gradients of the mean BCE loss into grads (same layout as params); the
// forward activations must be those of the same features and params
cudaError_t backward(const __nv_bfloat16* feat16, const float* label, __nv_bfloat16* const wb[4],
                     const __nv_bfloat16* act1, const __nv_bfloat16* act2,
                     const __nv_bfloat16* act3, const float* prob, __nv_bfloat16* g16, float* g32,
                     __nv_bfloat16* dz_a, __nv_bfloat16* dz_b, float* grads, float* loss_sum,
                     uint32_t W, uint32_t H, uint32_t* err, cudaStream_t st) {
  const uint32_t P = W * H;
  const float scale = 1.f / (float)P;
  const int rows_grid = (int)(H < (uint32_t)(num_sms() * 4) ? H : (uint32_t)(num_sms() * 4));
  cudaMemsetAsync(grads, 0, (size_t)(kOffB[3] + 1) * sizeof(float), st);
  cudaMemsetAsync(loss_sum, 0, sizeof(float), st);
  k_bce<<<num_sms() * 8, 256, 0, st>>>(prob, label, P, g16, g32, loss_sum);
  // layer 4: dW from g32 (one channel), data gradient into dz_a (masked by act3 > 0)
  k_wgrad<32, 1><<<rows_grid, 256, 0, st>>>(act3, 32, nullptr, g32, 1, W, H, scale,
                                             grads + kOffW[3], grads + kOffB[3]);
  cudaError_t e = launch_conv<16, 32, EPI_BWD_MASK_BF16>(g16, wb[3], nullptr, act3, dz_a, nullptr, W, H, err, st);
  if (e != cudaSuccess) return e;
  // layer 3
  k_wgrad<32, 32><<<rows_grid, 256, 0, st>>>(act2, 32, dz_a, nullptr, 32, W, H, scale,
                                              grads + kOffW[2], grads + kOffB[2]);
  e = launch_conv<32, 32, EPI_BWD_MASK_BF16>(dz_a, wb[2], nullptr, act2, dz_b, nullptr, W, H, err, st);
  if (e != cudaSuccess) return e;
  // layer 2
  k_wgrad<32, 32><<<rows_grid, 256, 0, st>>>(act1, 32, dz_b, nullptr, 32, W, H, scale,
                                              grads + kOffW[1], grads + kOffB[1]);
  e = launch_conv<32, 32, EPI_BWD_MASK_BF16>(dz_b, wb[1], nullptr, act1, dz_a, nullptr, W, H, err, st);
  if (e != cudaSuccess) return e;
  // layer 1 (no data gradient for the input features)
  k_wgrad<16, 32><<<rows_grid, 256, 0, st>>>(feat16, 9, dz_a, nullptr, 32, W, H, scale,
                                              grads + kOffW[0], grads + kOffB[0]);
  return cudaGetLastError();
}

cudaError_t adam(float* params, const float* grads, float* m, float* v, uint32_t n, float lr,
                 uint32_t step, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<(n + 255) / 256, 256, 0, st>>>(params, grads, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace nn
}  // namespace rt
