// Retrace-probability network: 4 layers of 3x3 convolutions
// (10 -> 32 -> 32 -> 32 -> 1, zero padding 1, ReLU, sigmoid), BF16 operands
// (E4M3 for layers 2-4 in FP8 inference) and FP32 accumulation on the
// 5th-generation tensor cores (sm_103a).
//
// Convolution as implicit GEMM on tcgen05 (k_conv_tma):
//   a persistent CTA computes tiles of R rows x W_t consecutive pixels:
//   output row ry is D_ry[128 pixels, Cout] = sum over the 9 taps (dy, dx) of
//   A(ry+dy, dx)[128, Cin] x B(dy, dx)[Cin, Cout], where A(h, dx) is halo row h
//   shifted by dx pixels. The input halo (R+2 rows of Cin channels) sits in
//   shared memory as 16-byte channel chunks ordered [chunk][halo pixel], so
//   every A(h, dx) is the same matrix shifted by h*pitch + dx rows: the
//   K-major, non-swizzled operand layout with 8-row core matrices 128 B apart
//   (SBO) and chunk planes (R+2)*pitch*16 B (rounded up to 128 B) apart (LBO).
//   Interleaved inputs (the 16-channel features) have 130-pixel halo rows and
//   W_t = 128; chunk-planar inputs (activations) are loaded as 2 KB box rows
//   of 128 pixels, W_t = 126 (the MMA lanes 126 and 127 read the next row and
//   are not stored).
//   Stacked taps: an MMA of N = Cout costs the tensor core as much as one of
//   N = 64 (about 45 cycles on GB300, measured; N = 96 about 56, N = 256 about
//   128, the full rate), so the three vertical taps of a kernel column are
//   multiplied in one MMA of N = 3 Cout: B(dx) = [B(2, dx) | B(1, dx) |
//   B(0, dx)], and A(h, dx) x B(dx) lands in TMEM at column h*Cout of the
//   tile's accumulators, where output row ry keeps its sum at column
//   (ry+2)*Cout: block j of the product (tap dy = 2 - j) adds into row h - dy.
//   Consecutive MMAs thus accumulate into overlapping column ranges (exact,
//   measured), (R+2) * 3 MMAs per K step and tile instead of R * 9; rows -2,
//   -1, R, R+1 of the accumulators take the products that fall outside the
//   tile and are never read. Every MMA accumulates; the epilogue zeroes the
//   columns it has read (and the four outside rows) before handing the
//   accumulators back. Weights are pre-packed in this stacked core-matrix
//   layout, [dx][chunk][3 Cout][chunk elements].
//   The CTA is warp-specialised: a TMA warp loads each tile's halo
//   (cp.async.bulk.tensor, zeros outside the image) into a ring of halo
//   buffers; an MMA warp issues the tile's MMAs (kind::f16 with BF16 inputs,
//   kind::f8f6f4 with E4M3) into one of two TMEM accumulator sets; the
//   epilogue warps read their TMEM lanes (tcgen05.ld 32x32b), hand the set
//   back and apply the fused epilogue (bias + ReLU -> BF16 or E4M3, bias +
//   sigmoid -> FP32, or the backward ReLU mask), so loads, MMAs and
//   epilogues of consecutive tiles overlap.
//   Every mbarrier wait has an iteration bound; on expiry the kernel sets the
//   error word, waits (bounded) for what it has in flight and frees its TMEM.
//
// Layouts in HBM: the 16-channel maps (network input features, the BCE
// gradient) are interleaved [P][16]; the 32-channel activations and data
// gradients are chunk-planar [4][P][8] BF16 or [2][P][16] E4M3 (plane k
// holds one 16-byte chunk of channels of every pixel), so a halo row of one
// chunk is one contiguous run and each warp's epilogue store a contiguous
// 512-byte run per plane.
//
// Backward pass: data gradients are convolutions with the 3x3 taps flipped
// and Cin/Cout swapped (same tensor-core kernel); weight gradients are an
// FP32 CUDA-core reduction over pixels; BCE on the sigmoid output; Adam on
// FP32 master weights.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdlib>

#include "rt_internal.cuh"

namespace rt {
namespace nn {

// Tuning knobs: RT_CONV_ROWS = image rows per tile (R accumulators of 128
// pixels share one halo of R+2 rows; with the stacked taps each accumulator
// set takes (R+4) * Cout TMEM columns, so R <= 4); RT_CONV_STAGES = the most
// halo buffers a CTA keeps (each layer takes as many as fit in ~220 KB of
// shared memory, up to this; the loads run that many tiles ahead of the MMAs).
// A halo load took ~5600 cycles to land at 1080p, two to three tiles' MMAs,
// yet deeper rings were slower: 3 / 4 / 5 / 6 / 8 stages, FP8 network at
// 1920x1080: 0.145 / 0.147 / 0.155 / 0.163 / 0.172 ms (3840x2160, 8 images:
// 0.398 / 0.397 / 0.426 / 0.434 ms per image for 3-6);
// RT_CONV_EPI_WG = epilogue warpgroups (4 warps each; group g takes the rows
// ry with ry % RT_CONV_EPI_WG == g of every tile; 4 groups were slower than 2:
// 0.197 against 0.147 ms, FP8 at 1920x1080).
#ifndef RT_CONV_ROWS
#define RT_CONV_ROWS 4
#endif
#ifndef RT_CONV_STAGES
#define RT_CONV_STAGES 4
#endif
#ifndef RT_CONV_EPI_WG
#define RT_CONV_EPI_WG 2
#endif
constexpr int kMaxStages = RT_CONV_STAGES;
static_assert(kMaxStages >= 2 && kMaxStages <= 8, "halo stages");
constexpr uint32_t kSmemBudget = 220u * 1024u;
constexpr int kEpiWarps = 4 * RT_CONV_EPI_WG;
constexpr int kConvTmaThreads = 32 * (kEpiWarps + 2);   // + the MMA warp and the TMA warp
constexpr int kRows = RT_CONV_ROWS;
constexpr int kTileM = 128;          // pixels per row tile (one MMA M block)
// The operand layout does not limit the MMAs: a 128-byte-swizzled operand
// costs what the non-swizzled one does (measured), and neither a halo whose odd
// chunks start a few pixels early (other shared-memory banks) nor swizzled
// weights changed the layered network's time.
constexpr int kHaloW = kTileM + 2;           // halo pixels per row of an interleaved input
// A planar (chunk-plane) input is loaded as one TMA box per chunk whose rows
// are 128 pixels x 16 bytes (256 8-byte elements, the largest box row), so
// its tiles are 126 output pixels wide (the MMA lanes 126 and 127 read the
// next halo row and are not stored). Boxes with rows of one 16-byte chunk
// make one 16-byte request per pixel that moves a whole 32-byte sector from
// L2: ~1500 requests per tile, whose transfer took longer than the tile's
// MMAs (measured).
constexpr int kHaloWPlanar = kTileM;
constexpr uint32_t kWaitBound = 1u << 26;

enum Epi : int { EPI_RELU_BF16 = 0, EPI_SIGMOID_F32 = 1, EPI_BWD_MASK_BF16 = 2, EPI_RELU_FP8 = 3 };

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// instruction descriptor: kind::f16, D = F32, A = B = BF16, both K-major
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Low and high words of a no-swizzle descriptor. A descriptor of the same
// operand at byte offset k from its base is the base's low word plus k >> 4
// (the start-address field cannot carry: shared addresses stay below 2^18),
// so the unrolled MMA loops below pay one integer add per descriptor.
__device__ __forceinline__ uint32_t desc_lo(uint32_t saddr, uint32_t lbo) {
  return ((saddr >> 4) & 0x3FFFu) | (((lbo >> 4) & 0x3FFFu) << 16);
}
__host__ __device__ constexpr uint32_t desc_hi(uint32_t sbo) {
  return ((sbo >> 4) & 0x3FFFu) | (1u << 14);   // bit 46 of the descriptor: tcgen05 version
}
__device__ __forceinline__ uint64_t desc_join(uint32_t lo, uint32_t hi) {
  return ((uint64_t)hi << 32) | lo;
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

// instruction descriptor: kind::f8f6f4, D = F32, A = B = E4M3 (format 0), both K-major
__host__ __device__ constexpr uint32_t make_idesc_e4m3(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// 4-D tiled TMA load of one box into shared memory, completion counted in
// bytes on the mbarrier; out-of-range elements are written as zeros
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// 5-D tiled TMA load (the same, with an image index among the coordinates)
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, int c4, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
      "r"(smem_u32(bar))
      : "memory");
}

// 16 consecutive TMEM columns of this warp's 32 lanes, without the wait:
// several loads share one tcgen05.wait::ld
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t r[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// All MMAs of one tile: for halo row h, kernel column dx and 32-byte K step
// ks (16 BF16 or 32 E4M3 channels), the halo shifted by h*130 + dx pixels
// times the stacked weights B(dx) (N = 3*COUT) accumulate into TMEM columns
// dtmem + h*COUT .. + 3*COUT - 1 (output rows h-2 .. h). kChunks = 16-byte
// channel chunks per pixel, kPlaneBytes = the distance between chunk planes
// of the halo, kPitch = pixels from one halo row to the next. The
// accumulators start at zero (cleared by the epilogue).
template <int kChunks, int COUT, uint32_t kPlaneBytes, int kPitch, bool FP8>
__device__ __forceinline__ void issue_tile_mmas(uint32_t hbase, uint32_t wbase, uint32_t dtmem,
                                                uint32_t idesc) {
  constexpr int kN = 3 * COUT;
  // A: LBO = the distance from an even chunk's core matrix to the odd one's;
  // B: chunk c + 1 of a weight row sits kN * 16 bytes after chunk c
  const uint32_t a_lo = desc_lo(hbase, kPlaneBytes), b_lo = desc_lo(wbase, kN * 16);
  constexpr uint32_t hi = desc_hi(128u);
#pragma unroll
  for (int h = 0; h < kRows + 2; ++h) {
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
      for (int ks = 0; ks < kChunks / 2; ++ks) {
        const uint32_t a_off = (2u * ks) * kPlaneBytes + (uint32_t)(h * kPitch + dx) * 16u;
        const uint32_t b_off = (uint32_t)((dx * kChunks + 2 * ks) * kN) * 16u;
        const uint64_t da = desc_join(a_lo + (a_off >> 4), hi), db = desc_join(b_lo + (b_off >> 4), hi);
        if (FP8) mma_e4m3(dtmem + (uint32_t)(h * COUT), da, db, idesc, 1u);
        else mma_bf16(dtmem + (uint32_t)(h * COUT), da, db, idesc, 1u);
      }
    }
  }
}

// zeroes 16 consecutive TMEM columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(
          taddr),
      "r"(0u)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------ conv kernel
// in:  BF16 [P][16] interleaved (CIN = 16) or [4][P][8] planar (CIN = 32);
//      with IN_FP8, E4M3 [2][P][16] planar (CIN = 32)
// wpk: packed weights, [dx][16-byte chunk][3 COUT: dy = 2, 1, 0][chunk elements]
//      (BF16 or E4M3)
// With IN_FP8 the accumulator of channel co is first multiplied by inv[co]
// (the product of the input's activation scale and the channel's weight
// scale, inverted: a power of two).
// EPI_RELU_BF16:     out (BF16 planar [4][P][8]) = relu(acc + bias)
// EPI_SIGMOID_F32:   out32[P] = sigmoid(acc[0] + bias[0])
// EPI_BWD_MASK_BF16: out (BF16 planar) = acc * (mask16 (planar) > 0)
// EPI_RELU_FP8:      out (E4M3 planar [2][P][16]) = e4m3(relu(acc + bias) * out_scale),
//                    round to nearest even, saturating at +-448
//
// Three roles. The last warp's first lane loads each tile's halo (one TMA box
// per 16-byte channel chunk, zeros outside the image) into a ring of
// RT_CONV_STAGES halo buffers, as far ahead as the ring allows; the warp
// before it issues the tile's MMAs into one of two TMEM accumulator sets as
// soon as its halo has landed and the epilogue has drained that set; the
// epilogue warps (RT_CONV_EPI_WG warpgroups; warp w reads TMEM lanes
// 32 (w % 4) .. +31) run the epilogue of tile i while the tensor cores work on
// tile i+1 and the TMA engine fetches the next tiles. Loads, MMAs and
// epilogues each wait only on their own barriers (in one thread, the loads'
// issue and the waits for their buffers held up the MMAs, measured).
//   halo_full[b]:  TMA bytes of halo buffer b arrived (expect_tx by the loader)
//   halo_empty[b]: the MMAs that read buffer b completed (tcgen05.commit)
//   acc_full[s]:   MMAs of accumulator set s done (tcgen05.commit)
//   acc_empty[s]:  every epilogue thread has read and zeroed set s
// Every wait is bounded; a wait that gives up sets the error word, and before
// the CTA frees TMEM and exits, the TMA warp waits (bounded) for the last copy
// into each buffer and the MMA warp for the MMAs it has issued.
template <int CIN, int COUT, bool IN_FP8, bool PLANAR>
struct ConvTmaLayout {
  static constexpr int kElem = IN_FP8 ? 1 : 2;                           // bytes per channel
  static constexpr int kChunks = CIN * kElem / 16;                       // 16-byte chunks per pixel
  static constexpr int kPitch = PLANAR ? kHaloWPlanar : kHaloW;          // halo pixels per row
  static constexpr int kOutW = kPitch - 2;                               // output pixels per row
  static constexpr uint32_t kBox = (uint32_t)(kRows + 2) * kPitch * 16u; // bytes of one TMA box
  static constexpr uint32_t kPlane = (kBox + 127u) & ~127u;            // chunk plane stride
  static constexpr uint32_t kHalo = ((kChunks * kPlane) + 1023u) & ~1023u;
  static constexpr uint32_t kWBytes = 9u * COUT * CIN * kElem;
  static constexpr uint32_t kW = (kWBytes + 127u) & ~127u;
  static constexpr uint32_t kAcc = (uint32_t)(kRows + 4) * COUT;       // rows -2 .. R+1
  static constexpr uint32_t kSet = kAcc <= 32 ? 32 : (kAcc <= 64 ? 64 : (kAcc <= 128 ? 128 : 256));
  static constexpr uint32_t kTmemCols = 2 * kSet;
  static constexpr uint32_t kFit = (kSmemBudget - kW - 1024u) / kHalo;   // halo buffers that fit
  static constexpr int kSt = kFit < 2u ? 2 : (kFit > (uint32_t)kMaxStages ? kMaxStages : (int)kFit);
  static constexpr size_t kSmem = kSt * (size_t)kHalo + kW + 64 * 4 + 20 * 8 + 16;
};

template <int CIN, int COUT, int EPI, bool PLANAR_IN, bool IN_FP8>
__global__ void __launch_bounds__(kConvTmaThreads, 1)
    k_conv_tma(const __grid_constant__ CUtensorMap tmap, const void* __restrict__ wpk,
               const float* __restrict__ bias, const float* __restrict__ inv,
               float out_scale, const __nv_bfloat16* __restrict__ mask16, void* __restrict__ out,
               float* __restrict__ out32, uint32_t W, uint32_t H, uint32_t n_img, uint32_t* err) {
  using Lt = ConvTmaLayout<CIN, COUT, IN_FP8, PLANAR_IN>;
  static_assert(CIN % 16 == 0 && (COUT == 16 || COUT == 32), "shape");
  static_assert(Lt::kTmemCols <= 512, "two accumulator sets must fit in TMEM");
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* halo0 = smem;
  unsigned char* wsm = smem + Lt::kSt * Lt::kHalo;
  float* bsm = reinterpret_cast<float*>(wsm + Lt::kW);    // bias[32], then inv[32]
  float* ism = bsm + 32;
  uint64_t* bars = reinterpret_cast<uint64_t*>(bsm + 64);
  uint64_t* halo_full = bars;        // [kSt]
  uint64_t* halo_empty = bars + 8;   // [kSt]
  uint64_t* acc_full = bars + 16;    // [2]
  uint64_t* acc_empty = bars + 18;   // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 20);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // n_img images of W x H pixels stacked in memory (image-major); a tile
  // never spans two images, and the halo rows outside its image read zeros
  const uint32_t tiles_x = (W + Lt::kOutW - 1) / Lt::kOutW;
  const uint32_t tiles_img = tiles_x * ((H + kRows - 1) / kRows);
  const uint32_t n_tiles = tiles_img * n_img;
  {
    const uint4* src = reinterpret_cast<const uint4*>(wpk);
    uint4* dst = reinterpret_cast<uint4*>(wsm);
    for (uint32_t i = tid; i < Lt::kWBytes / 16u; i += blockDim.x) dst[i] = src[i];
    if (tid < COUT) {
      bsm[tid] = bias ? bias[tid] : 0.f;
      ism[tid] = inv ? inv[tid] : 1.f;
    }
  }
  if (tid == 0) {
    for (int b = 0; b < Lt::kSt; ++b) {
      mbar_init(halo_full + b, 1);
      mbar_init(halo_empty + b, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full + b, 1);
      mbar_init(acc_empty + b, 32 * kEpiWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
  }
  if (warp == 0) tmem_alloc(tslot, Lt::kTmemCols);
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  // the MMAs only accumulate: clear both accumulator sets once (warp w % 4
  // may address TMEM lanes 32 (w % 4) .. +31)
  if (warp < 4) {
    for (uint32_t c = 0; c < Lt::kTmemCols; c += 16) tmem_zero16(tmem + ((uint32_t)(warp * 32) << 16) + c);
    tmem_wait_st();
  }
  fence_before();
  __syncthreads();
  fence_after();

  const uint32_t my_tiles = blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (warp == kEpiWarps) {
    // ---- MMA issue: tile it of this CTA's sequence reads halo buffer it % kSt
    if (lane == 0) {
      const uint32_t idesc = IN_FP8 ? make_idesc_e4m3(kTileM, 3 * COUT) : make_idesc(kTileM, 3 * COUT);
      const uint32_t wbase = smem_u32(wsm);
      bool issued_acc[2] = {false, false}, issued_he[Lt::kSt];
      uint32_t acc_par[2] = {0, 0}, he_par[Lt::kSt];     // parity of the last commit
#pragma unroll
      for (int b = 0; b < Lt::kSt; ++b) { issued_he[b] = false; he_par[b] = 0; }
      bool ok = true;
      for (uint32_t it = 0; it < my_tiles; ++it) {
        const int b = (int)(it % Lt::kSt), sa = (int)(it & 1u);
        if (!mbar_wait(halo_full + b, (it / Lt::kSt) & 1u)) { ok = false; break; }
        if (it >= 2 && !mbar_wait(acc_empty + sa, ((it >> 1) - 1) & 1u)) { ok = false; break; }
        fence_after();
        issue_tile_mmas<Lt::kChunks, COUT, Lt::kPlane, Lt::kPitch, IN_FP8>(
            smem_u32(halo0 + (size_t)b * Lt::kHalo), wbase, tmem + (uint32_t)sa * Lt::kSet, idesc);
        mma_commit(halo_empty + b);   // the buffer may be reloaded once these MMAs completed
        mma_commit(acc_full + sa);
        issued_he[b] = true;
        he_par[b] = (it / Lt::kSt) & 1u;
        issued_acc[sa] = true;
        acc_par[sa] = (it >> 1) & 1u;
      }
      if (!ok) atomicOr(err, ERR_ITER);
      // drain: the MMAs issued here complete (and signal) before TMEM is freed
      for (int b = 0; b < 2; ++b)
        if (issued_acc[b]) mbar_wait(acc_full + b, acc_par[b]);
      for (int b = 0; b < Lt::kSt; ++b)
        if (issued_he[b]) mbar_wait(halo_empty + b, he_par[b]);
    }
    __syncwarp();
  } else if (warp == kEpiWarps + 1) {
    // ---- TMA loads: tile j into buffer j % kSt once the MMAs of tile
    // j - kSt (the buffer's previous tile) completed
    if (lane == 0) {
      bool ok = true;
      uint32_t n_loaded = 0;
      for (uint32_t j = 0; j < my_tiles; ++j) {
        const int b = (int)(j % Lt::kSt);
        if (j >= (uint32_t)Lt::kSt && !mbar_wait(halo_empty + b, ((j / Lt::kSt) - 1) & 1u)) { ok = false; break; }
        const uint32_t tile = blockIdx.x + j * gridDim.x;
        const int img = (int)(tile / tiles_img);
        const uint32_t it_img = tile - (uint32_t)img * tiles_img;
        const int ty = (int)(it_img / tiles_x);
        const int y = ty * kRows, x0 = (int)(it_img - (uint32_t)ty * tiles_x) * Lt::kOutW;
        mbar_arrive_expect_tx(halo_full + b, (uint32_t)Lt::kChunks * Lt::kBox);
#pragma unroll
        for (int c = 0; c < Lt::kChunks; ++c) {
          unsigned char* plane = halo0 + (size_t)b * Lt::kHalo + (size_t)c * Lt::kPlane;
          if (PLANAR_IN)   // tensor {8-byte halves of pixels (2 W), H, images, chunks}
            tma_load_4d(plane, &tmap, 2 * (x0 - 1), y - 1, img, c, halo_full + b);
          else             // tensor {16 B of channels, chunks, W, H, images}
            tma_load_5d(plane, &tmap, 0, c, x0 - 1, y - 1, img, halo_full + b);
        }
        n_loaded = j + 1;
      }
      if (!ok) atomicOr(err, ERR_ITER);
      // drain: the last copy into each buffer has landed before the CTA exits
      for (uint32_t j = n_loaded > (uint32_t)Lt::kSt ? n_loaded - Lt::kSt : 0; j < n_loaded; ++j)
        mbar_wait(halo_full + (j % Lt::kSt), (j / Lt::kSt) & 1u);
    }
    __syncwarp();
  } else {
    // Each epilogue warp first copies its rows of the accumulator set into
    // registers, zeroes them (and group 0 the rows outside the tile) and hands
    // the set back, so the next tile's MMAs start while it converts and
    // stores: the tensor core then waits only for the TMEM reads, not for the
    // whole epilogue.
    constexpr int kMine = kRows / RT_CONV_EPI_WG;   // rows per epilogue warp
    constexpr int kHalves = COUT / 16;
    static_assert(kRows % RT_CONV_EPI_WG == 0, "rows per tile must split evenly over the epilogue groups");
    const int quarter = warp & 3, group = warp >> 2;   // TMEM lanes 32*quarter .. +31
    const size_t P = (size_t)W * H * n_img;            // pixels of a channel plane
    // per output channel c: out = max(fma(acc, sc[c], bi[c]), 0) (or the
    // sigmoid of it), with the input's inverse scale (E4M3 inputs) and the
    // output scale (E4M3 outputs) folded in: all are powers of two, so the
    // folded form rounds exactly like scaling the rounded sum
    float sc[COUT], bi[COUT];
#pragma unroll
    for (int c = 0; c < COUT; ++c) {
      const float os = EPI == EPI_RELU_FP8 ? out_scale : 1.f;
      sc[c] = (IN_FP8 ? ism[c] : 1.f) * os;
      bi[c] = bsm[c] * os;
    }
    uint32_t it = 0;
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
      const int s = (int)(it & 1u);
      // warp-uniform outcome: tcgen05.ld below is a warp-collective instruction
      if (!__all_sync(0xFFFFFFFFu, mbar_wait(acc_full + s, (it >> 1) & 1u))) {
        if (lane == 0) atomicOr(err, ERR_ITER);
        break;
      }
      fence_after();
      // output row ry's sums sit in columns (ry + 2) * COUT of the set
      const uint32_t set_addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)s * Lt::kSet;
      uint32_t r[kMine][kHalves][16];
#pragma unroll
      for (int k = 0; k < kMine; ++k)
#pragma unroll
        for (int half = 0; half < kHalves; ++half)
          tmem_ld16_nowait(set_addr + (uint32_t)((group + k * RT_CONV_EPI_WG + 2) * COUT + half * 16), r[k][half]);
      tmem_wait_ld();
#pragma unroll
      for (int k = 0; k < kMine; ++k)
#pragma unroll
        for (int half = 0; half < kHalves; ++half)
          tmem_zero16(set_addr + (uint32_t)((group + k * RT_CONV_EPI_WG + 2) * COUT + half * 16));
      if (group == 0) {   // rows -2, -1, R, R+1
#pragma unroll
        for (int c = 0; c < 2 * COUT; c += 16) {
          tmem_zero16(set_addr + (uint32_t)c);
          tmem_zero16(set_addr + (uint32_t)((kRows + 2) * COUT + c));
        }
      }
      tmem_wait_st();
      fence_before();
      mbar_arrive(acc_empty + s);

      const uint32_t img = tile / tiles_img;
      const uint32_t it_img = tile - img * tiles_img;
      const int ty = (int)(it_img / tiles_x);
      const int y = ty * kRows;
      const int x0 = (int)(it_img - (uint32_t)ty * tiles_x) * Lt::kOutW;
      const int x = x0 + quarter * 32 + lane;
      const bool lane_ok = quarter * 32 + lane < Lt::kOutW;
#pragma unroll
      for (int k = 0; k < kMine; ++k) {
        const int yy = y + group + k * RT_CONV_EPI_WG;
        if (!(lane_ok && x < (int)W && yy < (int)H)) continue;
        const size_t p = ((size_t)img * H + yy) * W + x;
        if (EPI == EPI_SIGMOID_F32) {
          const float z = fmaf(__uint_as_float(r[k][0][0]), sc[0], bi[0]);
          out32[p] = 1.f / (1.f + __expf(-z));
        } else if (EPI == EPI_RELU_FP8) {
#pragma unroll
          for (int half = 0; half < kHalves; ++half) {
            uint32_t packed[4];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int c0 = half * 16 + 2 * i, c1 = c0 + 1;
              const float a0 = __uint_as_float(r[k][half][2 * i]), a1 = __uint_as_float(r[k][half][2 * i + 1]);
              const float y0 = fmaxf(fmaf(a0, sc[c0], bi[c0]), 0.f);
              const float y1 = fmaxf(fmaf(a1, sc[c1], bi[c1]), 0.f);
              const uint32_t q = __nv_cvt_float2_to_fp8x2(make_float2(y0, y1), __NV_SATFINITE, __NV_E4M3);
              if (i & 1) packed[i >> 1] |= q << 16; else packed[i >> 1] = q;
            }
            // E4M3 planar: plane `half` holds channels 16 half .. 16 half + 15
            *reinterpret_cast<uint4*>(static_cast<uint8_t*>(out) + (half * P + p) * 16) =
                make_uint4(packed[0], packed[1], packed[2], packed[3]);
          }
        } else {
          __nv_bfloat16* out16 = static_cast<__nv_bfloat16*>(out);
#pragma unroll
          for (int half = 0; half < kHalves; ++half) {
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[k][half][i]);
            uint32_t packed[8];
            if (EPI == EPI_RELU_BF16) {
#pragma unroll
              for (int i = 0; i < 8; ++i)
                packed[i] = pack_bf16(fmaxf(v[2 * i] + bi[half * 16 + 2 * i], 0.f),
                                      fmaxf(v[2 * i + 1] + bi[half * 16 + 2 * i + 1], 0.f));
            } else {
              // planar: channels 16 half + 0..7 and + 8..15 sit in planes 2 half, 2 half + 1
              const uint4 ma = *reinterpret_cast<const uint4*>(mask16 + ((2 * half) * P + p) * 8);
              const uint4 mb = *reinterpret_cast<const uint4*>(mask16 + ((2 * half + 1) * P + p) * 8);
              const uint32_t mw[8] = {ma.x, ma.y, ma.z, ma.w, mb.x, mb.y, mb.z, mb.w};
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const __nv_bfloat162 mm = *reinterpret_cast<const __nv_bfloat162*>(&mw[i]);
                const float m0 = __bfloat162float(mm.x), m1 = __bfloat162float(mm.y);
                packed[i] = pack_bf16(m0 > 0.f ? v[2 * i] : 0.f, m1 > 0.f ? v[2 * i + 1] : 0.f);
              }
            }
            *reinterpret_cast<uint4*>(out16 + ((2 * half) * P + p) * 8) =
                make_uint4(packed[0], packed[1], packed[2], packed[3]);
            *reinterpret_cast<uint4*>(out16 + ((2 * half + 1) * P + p) * 8) =
                make_uint4(packed[4], packed[5], packed[6], packed[7]);
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, Lt::kTmemCols);
}


// ------------------------------------------------ weight packing (FP32 -> BF16)
// Canonical parameter layout of a layer: W[Cout][Cin][3][3] then b[Cout].
// Packed (k_conv_tma's stacked taps): element i of a conv with output
// channels cout_p and input channels cin_p, chunks of `per` elements, is
// [dx][ci / per][j * cout_p + co][ci % per] with tap (dy = 2 - j, dx).
struct StackedIndex {
  int co, ci, tap;
};
__device__ __forceinline__ StackedIndex stacked_index(int i, int per, int cout_p, int cin_p) {
  const int e = i % per, rest = i / per;
  const int n = rest % (3 * cout_p), rest2 = rest / (3 * cout_p);
  const int chunk = rest2 % (cin_p / per), dx = rest2 / (cin_p / per);
  const int j = n / cout_p;
  return {n - j * cout_p, chunk * per + e, (2 - j) * 3 + dx};
}

// forward pack: W[co][ci][tap] with ci < cin_pad, co < cout_pad (zero fill)
__global__ void k_pack_fwd(const float* __restrict__ Wt, int cout, int cin, int cout_pad,
                           int cin_pad, __nv_bfloat16* __restrict__ out) {
  const int n = 9 * cin_pad * cout_pad;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const StackedIndex x = stacked_index(i, 8, cout_pad, cin_pad);
    float v = 0.f;
    if (x.co < cout && x.ci < cin) v = Wt[((size_t)x.co * cin + x.ci) * 9 + x.tap];
    out[i] = __float2bfloat16_rn(v);
  }
}

// backward-data pack: a conv whose output channel o is forward input channel
// ci and whose input channel c is forward output channel co, taps flipped:
// W'[o][c][tap] = W[c][o][8 - tap]
__global__ void k_pack_bwd(const float* __restrict__ Wt, int cout, int cin, int cout_pad,
                           int cin_pad, __nv_bfloat16* __restrict__ out) {
  // as a conv: CIN' = cout_pad, COUT' = cin_pad
  const int n = 9 * cout_pad * cin_pad;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const StackedIndex x = stacked_index(i, 8, cin_pad, cout_pad);   // x.co: forward ci, x.ci: forward co
    float v = 0.f;
    if (x.ci < cout && x.co < cin) v = Wt[((size_t)x.ci * cin + x.co) * 9 + (8 - x.tap)];
    out[i] = __float2bfloat16_rn(v);
  }
}

// FP8 forward pack of layers 2-4: E4M3 of W[co][ci][tap] * scale[co] (round
// to nearest even, saturating), chunks of 16 elements, zero fill
__global__ void k_pack_fwd_fp8(const float* __restrict__ Wt, int cout, int cin, int cout_pad,
                               int cin_pad, const float* __restrict__ scale, uint8_t* __restrict__ out) {
  const int n = 9 * cin_pad * cout_pad;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const StackedIndex x = stacked_index(i, 16, cout_pad, cin_pad);
    float v = 0.f;
    if (x.co < cout && x.ci < cin) v = Wt[((size_t)x.co * cin + x.ci) * 9 + x.tap] * scale[x.co];
    out[i] = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
  }
}

// largest element of a non-negative BF16 map (ReLU outputs): float bits of
// non-negative values order like unsigned integers
__global__ void k_amax(const __nv_bfloat16* __restrict__ a, size_t n, unsigned* __restrict__ out) {
  float m = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, __bfloat162float(a[i]));
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_down_sync(0xFFFFFFFFu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
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
// dW[co][ci][ky][kx] = scale * sum_x dZ[y][x][co] * A[y+ky-1][x+kx-1][ci],
// db[co] = scale * sum_x dZ[y][x][co]; each CTA takes every gridDim.x-th image
// row, a 64-pixel chunk at a time through shared memory, FP32 accumulation,
// and writes its unscaled partial sums (canonical layout: the layer's weights
// then its biases) to its own row of `part`; k_wgrad_reduce then adds the
// rows in a fixed order, so the gradient -- and training -- is the same bit
// for bit from run to run (atomics would add the CTAs in arrival order).
// A is interleaved [P][16] when CIN_PAD = 16 (the input features) and planar
// [4][P][8] when CIN_PAD = 32 (activations); dZ comes as FP32 (layer 4, one
// channel) or as a planar 32-channel BF16 map.
template <int CIN_PAD, int COUT>
__global__ void __launch_bounds__(256) k_wgrad(const __nv_bfloat16* __restrict__ A, int cin,
                                               const __nv_bfloat16* __restrict__ dz16,
                                               const float* __restrict__ dz32, uint32_t W,
                                               uint32_t H, float* __restrict__ part) {
  const size_t P = (size_t)W * H;
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
          v = __bfloat162float(CIN_PAD == 32
                                   ? A[((size_t)(c >> 3) * P + (size_t)gy * W + gx) * 8 + (c & 7)]
                                   : A[((size_t)gy * W + gx) * CIN_PAD + c]);
        sA[dy][xx][c] = v;
      }
      for (int k = tid; k < kChunk * COUT; k += 256) {
        const int co = k % COUT, xx = k / COUT;
        const uint32_t gx = x0 + xx;
        float v = 0.f;
        if (gx < W) {
          const size_t p = (size_t)y * W + gx;
          v = dz32 ? dz32[p] : __bfloat162float(dz16[((size_t)(co >> 3) * P + p) * 8 + (co & 7)]);
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
  const size_t n_w = (size_t)COUT * cin * 9;
  float* row = part + (size_t)blockIdx.x * (n_w + COUT);
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int o = tid + i * 256;
    if (o < kOut) {
      const int tap = o % 9, rest = o / 9;
      const int ci = rest % CIN_PAD, co = rest / CIN_PAD;
      if (ci < cin) row[((size_t)co * cin + ci) * 9 + tap] = acc[i];
    }
  }
  if (tid < COUT) row[n_w + tid] = bacc;
}

// out[j] = scale * sum over b = 0 .. nblk-1 of part[b][j], in a fixed order:
// warp w of a block adds rows w, w + 8, w + 16, ... of 32 consecutive
// columns, then thread 0..31 adds the 8 warp sums in warp order.
__global__ void __launch_bounds__(256) k_wgrad_reduce(const float* __restrict__ part, uint32_t nblk,
                                                      uint32_t n, float scale, float* __restrict__ out) {
  __shared__ float s[8][32];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t j = blockIdx.x * 32 + lane;
  float a = 0.f;
  if (j < n)
    for (uint32_t b = warp; b < nblk; b += 8) a += part[(size_t)b * n + j];
  s[warp][lane] = a;
  __syncthreads();
  if (warp == 0 && j < n) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += s[w][lane];
    out[j] = t * scale;
  }
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

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependency on libcuda)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// Tensor map of a BF16 or E4M3 map for the halo boxes of k_conv_tma.
// Interleaved [images][H][W][C] is viewed as {chunk elements, chunks, W, H,
// images} with one box {chunk elements, 1, 130, R+2, 1} per chunk; planar
// [chunks][images][H][W][16 bytes] as 8-byte elements {2 W, H, images,
// chunks} with one box {256 (128 pixels), R+2, 1, 1} per chunk.
template <int CIN, bool PLANAR, bool FP8>
cudaError_t make_halo_map(CUtensorMap* map, const void* in, uint32_t W, uint32_t H, uint32_t n_img) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn) return cudaErrorNotSupported;
  if (reinterpret_cast<uintptr_t>(in) & 15u) return cudaErrorInvalidValue;
  constexpr int kElem = FP8 ? 1 : 2, kPer = 16 / kElem, kChunks = CIN / kPer;
  const cuuint64_t P = (cuuint64_t)W * H;
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult r;
  if (PLANAR) {
    const cuuint64_t d[4] = {2ull * W, H, n_img, kChunks};
    const cuuint64_t st[3] = {(cuuint64_t)W * 16, P * 16, P * n_img * 16};
    const cuuint32_t bx[4] = {2u * kHaloWPlanar, (cuuint32_t)(kRows + 2), 1, 1};
    r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<void*>(in), d, st, bx, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    const cuuint64_t d[5] = {kPer, kChunks, W, H, n_img};
    const cuuint64_t st[4] = {16, (cuuint64_t)CIN * kElem, (cuuint64_t)W * CIN * kElem,
                              P * CIN * kElem};
    const cuuint32_t bx[5] = {kPer, 1, (cuuint32_t)kHaloW, (cuuint32_t)(kRows + 2), 1};
    r = fn(map, FP8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5,
           const_cast<void*>(in), d, st, bx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// in: BF16 interleaved [P][16] when CIN = 16, BF16 planar [4][P][8] when
// CIN = 32, E4M3 planar [2][P][16] with IN_FP8
template <int CIN, int COUT, int EPI, bool IN_FP8 = false>
cudaError_t launch_conv(const void* in, const void* wpk, const float* bias, const float* inv,
                        float out_scale, const __nv_bfloat16* mask16, void* out, float* out32,
                        uint32_t W, uint32_t H, uint32_t* err, cudaStream_t st, uint32_t n_img = 1) {
  constexpr bool kPlanarIn = IN_FP8 || CIN == 32;
  using Lt = ConvTmaLayout<CIN, COUT, IN_FP8, kPlanarIn>;
  const uint32_t tiles = ((W + Lt::kOutW - 1) / Lt::kOutW) * ((H + kRows - 1) / kRows) * n_img;
  size_t smem = Lt::kSmem + (size_t)(g_conv_smem_pad + conv_smem_pad());
  // a CTA that takes all 512 TMEM columns must be alone on its SM: ask for
  // more than half of the SM's shared memory so a second one cannot be placed
  if (Lt::kTmemCols == 512 && smem < 116u * 1024u) smem = 116u * 1024u;
  static size_t configured = 0;
  if (configured < smem) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_tma<CIN, COUT, EPI, kPlanarIn, IN_FP8>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  CUtensorMap map;
  cudaError_t e = make_halo_map<CIN, kPlanarIn, IN_FP8>(&map, in, W, H, n_img);
  if (e != cudaSuccess) return e;
  // resident CTAs per SM from the shared-memory footprint (227 KB usable,
  // 1 KB reserved per CTA) and the TMEM columns (512 per SM) each CTA takes
  int per_sm = (int)((227u * 1024u) / (smem + 1024u));
  if (per_sm > (int)(512 / Lt::kTmemCols)) per_sm = (int)(512 / Lt::kTmemCols);
  if (per_sm < 1) per_sm = 1;
  uint32_t grid = (uint32_t)(num_sms() * per_sm);
  if (grid > tiles) grid = tiles;
  k_conv_tma<CIN, COUT, EPI, kPlanarIn, IN_FP8><<<grid, kConvTmaThreads, smem, st>>>(
      map, wpk, bias, inv, out_scale, mask16, out, out32, W, H, n_img, err);
  return cudaGetLastError();
}
}  // namespace

void set_conv_smem_pad(int bytes) { g_conv_smem_pad = bytes; }

// parameter offsets (canonical layout W[Cout][Cin][3][3], b[Cout] per layer)
constexpr uint32_t kOffW[4] = {0, 2912, 12160, 21408};
constexpr uint32_t kOffB[4] = {2880, 12128, 21376, 21696};
constexpr int kCout[4] = {32, 32, 32, 1};
constexpr int kCin[4] = {10, 32, 32, 32};
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
                    uint32_t W, uint32_t H, uint32_t* err, cudaStream_t st, uint32_t n_img) {
  cudaError_t e;
  e = launch_conv<16, 32, EPI_RELU_BF16>(feat16, wf[0], params + kOffB[0], nullptr, 1.f, nullptr, act1,
                                         nullptr, W, H, err, st, n_img);
  if (e != cudaSuccess) return e;
  e = launch_conv<32, 32, EPI_RELU_BF16>(act1, wf[1], params + kOffB[1], nullptr, 1.f, nullptr, act2,
                                         nullptr, W, H, err, st, n_img);
  if (e != cudaSuccess) return e;
  e = launch_conv<32, 32, EPI_RELU_BF16>(act2, wf[2], params + kOffB[2], nullptr, 1.f, nullptr, act3,
                                         nullptr, W, H, err, st, n_img);
  if (e != cudaSuccess) return e;
  return launch_conv<32, 16, EPI_SIGMOID_F32>(act3, wf[3], params + kOffB[3], nullptr, 1.f, nullptr,
                                             nullptr, prob, W, H, err, st, n_img);
}

cudaError_t pack_weights_fp8(const float* params, const float* const scale[3], uint8_t* const w8[3],
                             cudaStream_t st) {
  for (int l = 1; l < 4; ++l)
    k_pack_fwd_fp8<<<64, 256, 0, st>>>(params + kOffW[l], kCout[l], kCin[l], kCoutPad[l], kCinPad[l],
                                       scale[l - 1], w8[l - 1]);
  return cudaGetLastError();
}

size_t packed_fp8_bytes(int l) { return 9ull * kCinPad[l] * kCoutPad[l]; }

// the FP8 network: layer 1 in BF16 with E4M3 output, layers 2-4 on E4M3
// operands (kind::f8f6f4); act8 buffers hold E4M3 planar [2][P][16]
cudaError_t forward_fp8(const __nv_bfloat16* feat16, const float* params, __nv_bfloat16* const wf[4],
                        uint8_t* const w8[3], const float* const inv[3], const float act_scale[3],
                        uint8_t* act8_1, uint8_t* act8_2, uint8_t* act8_3, float* prob, uint32_t W,
                        uint32_t H, uint32_t* err, cudaStream_t st, uint32_t n_img) {
  cudaError_t e;
  e = launch_conv<16, 32, EPI_RELU_FP8>(feat16, wf[0], params + kOffB[0], nullptr, act_scale[0], nullptr,
                                        act8_1, nullptr, W, H, err, st, n_img);
  if (e != cudaSuccess) return e;
  e = launch_conv<32, 32, EPI_RELU_FP8, true>(act8_1, w8[0], params + kOffB[1], inv[0], act_scale[1],
                                              nullptr, act8_2, nullptr, W, H, err, st, n_img);
  if (e != cudaSuccess) return e;
  e = launch_conv<32, 32, EPI_RELU_FP8, true>(act8_2, w8[1], params + kOffB[2], inv[1], act_scale[2],
                                              nullptr, act8_3, nullptr, W, H, err, st, n_img);
  if (e != cudaSuccess) return e;
  return launch_conv<32, 16, EPI_SIGMOID_F32, true>(act8_3, w8[2], params + kOffB[3], inv[2], 1.f, nullptr,
                                                    nullptr, prob, W, H, err, st, n_img);
}

// raises amax3[l] to the largest value of hidden activation l (the caller
// clears amax3 before the first map it measures)
cudaError_t activation_amax(const __nv_bfloat16* const act[3], uint64_t P, unsigned* amax3,
                            cudaStream_t st) {
  for (int l = 0; l < 3; ++l) k_amax<<<num_sms() * 4, 256, 0, st>>>(act[l], P * 32, amax3 + l);
  return cudaGetLastError();
}

// gradients of the mean BCE loss into grads (same layout as params); the
// forward activations must be those of the same features and params
cudaError_t backward(const __nv_bfloat16* feat16, const float* label, __nv_bfloat16* const wb[4],
                     const __nv_bfloat16* act1, const __nv_bfloat16* act2,
                     const __nv_bfloat16* act3, const float* prob, __nv_bfloat16* g16, float* g32,
                     __nv_bfloat16* dz_a, __nv_bfloat16* dz_b, float* wpart, float* grads,
                     float* loss_sum, uint32_t W, uint32_t H, uint32_t* err, cudaStream_t st) {
  const uint32_t P = W * H;
  const float scale = 1.f / (float)P;
  const int rows_grid = wgrad_blocks(H);
  // weight gradient of layer l from its per-CTA partial sums (fixed order)
  auto reduce = [&](int l) {
    const uint32_t n = (uint32_t)kCout[l] * (uint32_t)kCin[l] * 9u + (uint32_t)kCout[l];
    k_wgrad_reduce<<<(n + 31) / 32, 256, 0, st>>>(wpart, (uint32_t)rows_grid, n, scale, grads + kOffW[l]);
  };
  cudaMemsetAsync(loss_sum, 0, sizeof(float), st);
  k_bce<<<num_sms() * 8, 256, 0, st>>>(prob, label, P, g16, g32, loss_sum);
  // layer 4: dW from g32 (one channel), data gradient into dz_a (masked by act3 > 0)
  k_wgrad<32, 1><<<rows_grid, 256, 0, st>>>(act3, 32, nullptr, g32, W, H, wpart);
  reduce(3);
  cudaError_t e = launch_conv<16, 32, EPI_BWD_MASK_BF16>(g16, wb[3], nullptr, nullptr, 1.f, act3, dz_a,
                                                         nullptr, W, H, err, st);
  if (e != cudaSuccess) return e;
  // layer 3
  k_wgrad<32, 32><<<rows_grid, 256, 0, st>>>(act2, 32, dz_a, nullptr, W, H, wpart);
  reduce(2);
  e = launch_conv<32, 32, EPI_BWD_MASK_BF16>(dz_a, wb[2], nullptr, nullptr, 1.f, act2, dz_b, nullptr,
                                             W, H, err, st);
  if (e != cudaSuccess) return e;
  // layer 2
  k_wgrad<32, 32><<<rows_grid, 256, 0, st>>>(act1, 32, dz_b, nullptr, W, H, wpart);
  reduce(1);
  e = launch_conv<32, 32, EPI_BWD_MASK_BF16>(dz_b, wb[1], nullptr, nullptr, 1.f, act1, dz_a, nullptr,
                                             W, H, err, st);
  if (e != cudaSuccess) return e;
  // layer 1 (no data gradient for the input features)
  k_wgrad<16, 32><<<rows_grid, 256, 0, st>>>(feat16, kCin[0], dz_a, nullptr, W, H, wpart);
  reduce(0);
  return cudaGetLastError();
}

int wgrad_blocks(uint32_t H) { return (int)(H < (uint32_t)(num_sms() * 4) ? H : (uint32_t)(num_sms() * 4)); }

size_t wgrad_part_floats(uint32_t H) { return (size_t)wgrad_blocks(H) * (32u * 32u * 9u + 32u); }

cudaError_t adam(float* params, const float* grads, float* m, float* v, uint32_t n, float lr,
                 uint32_t step, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<(n + 255) / 256, 256, 0, st>>>(params, grads, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace nn
}  // namespace rt
