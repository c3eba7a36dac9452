// Stereo-pair ray tracing on the GPU (sm_103a): the hot path.
//
// Paper Sec. 3: the left and right channel are independent ("parallel level
// 1") and the pixels of a channel are traced in parallel ("parallel level 2");
// the image is split into parts processed by parallel workers (Figure 1).
// Here both eyes share one persistent launch and one warp: a warp pulls a
// tile of 4x4 pixels from a global counter and traces it for both eyes, the
// two rays of a pixel in neighbouring lanes, so the eyes' nearly identical
// rays fetch the same BVH nodes in the same load and their shadow and mirror
// rays queue side by side (1080p blob pair: 1.143 -> 1.042 ms against 8x4
// tiles of one eye, eyes alternating between warps). Renders of one eye, and
// of scenes of fewer than kPairEyesPrims primitives, use those 8x4 tiles.
//
// Per stereo pair:
//   k_render   one persistent kernel. Every warp owns two small wavefront
//              queues in global memory (L2-resident): shadow rays and mirror
//              rays produced by its own shading. Each round the warp picks,
//              warp-uniformly, 32 queued shadow rays (any-hit), else 32
//              queued mirror rays (closest hit + shade), else a new primary
//              tile (generate + closest hit + shade). Once every tile has
//              been handed out, a warp hands its whole queue to two global
//              drain pools (shadow, mirror) and from then on takes batches
//              of up to 32 rays from the pools, mirror rays first, handing
//              back whatever its shading queues: the rest of the frame
//              spreads over every warp still running, in full rounds,
//              instead of each warp tracing its own backlog alone (measured
//              on the 1080p blob pair: 1.52 -> 1.30 ms). No ray waits for
//              a later launch, and there is one launch tail per frame
//              instead of one per bounce depth.
//   k_resolve  fixed-point sums -> float RGB, clamp to [0,1]
//
// Colour sums are fixed-point uint32 per channel (round(value * 2^k); the
// primary ray stores its term, every later ray adds its own atomically):
// integer addition is associative, so the image does not depend on the order
// in which shadow rays finish, and both eyes of a zero-separation pair are
// bitwise identical.
//
// Traversal (Table 1 of the paper: BVH trees): BVH2 nodes of 64 B with both
// child boxes, read as four 16-byte vector loads through the read-only path;
// slab tests in FP32 with fused multiply-adds and three-input min/max; the
// far child is pushed on a per-thread stack of 64 entries, the near child is
// visited first. The tree is the SAH rebuild of the scene's LBVH (sah.cu,
// depth <= 60 by its depth budget) or the LBVH itself (depth <= 64: a radix
// tree over unique 64-bit keys). Each loop has an iteration bound and the
// stack a size check; hitting either sets the error word.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_internal.cuh"
#include "trace_dev.cuh"

namespace rt {
namespace {

struct KParams {
  RenderArgs a;
  uint32_t* accum;
  float4* wq;          // warp queues: per warp cap_s shadow then cap_r mirror entries
  float4* pool;        // drain pools: cap_p shadow entries, then cap_p mirror entries
  uint32_t* pool_flag; // per pool entry: epoch of the render that wrote it
  uint32_t* counters;
  uint32_t cap_s, cap_r, cap_p;
  uint32_t epoch;      // this render's epoch (> 0)
  uint32_t n_tiles;    // primary tiles of 32 rays (pixel list: 32 entries each)
  bool share_partial;  // drain: hand over backlogs of less than a round too
  bool pair_eyes;      // primary tiles of 4x4 pixels of both eyes (else 8x4 of one eye)
  uint32_t n_frames;   // frames traced by this launch (each its own camera, same image size)
  uint32_t tiles_pf;   // primary tiles per frame
  CameraParams cams[kMaxFrames];   // the camera of each frame (cams[0] = a.cam)
};

constexpr uint32_t kNullPix = 0xFFFFFFFFu;   // pool entry that carries no ray
constexpr uint32_t kSpinMax = 1u << 22;        // bound of every wait on another warp
// scenes of at least this many primitives hand over partial backlogs too
// (1080p blob pair, 257k primitives: 1.301 ms sharing everything, 1.330
// keeping partial backlogs; small scene, 10 primitives: 0.262 against 0.239)
constexpr uint32_t kSharePartialPrims = 1024;
// scenes of at least this many primitives trace both eyes of a pixel in one
// warp; in smaller ones the walks are a few nodes long and 8x4 tiles of one
// eye, eyes alternating between warps, are faster (polyhedra of 12-180
// triangles at 1080p: 5-9 % with one or two lights)
constexpr uint32_t kPairEyesPrims = 1024;

// Polls use relaxed (L2-coherent) loads: an acquire load would invalidate
// the SM's L1, which holds the top of the BVH for every warp on the SM. A
// pool entry is read after its flag has been seen (a control dependency) with
// L2 loads, and its producer publishes the flag with a release store.
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int2 ld_volatile2(const uint32_t* p) {
  int2 v;
  asm volatile("ld.volatile.global.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p) : "memory");
  return v;
}
// Drain pool protocol (one lane of a warp calls these; every step is one
// atomic, no retry loop, so thousands of warps can hand over and take at
// once): a warp reserves entries with an add on the tail, writes them and
// sets each entry's flag to the render's epoch, then adds their number to
// `avail`. A taker first claims up to 32 from `avail` (a counting semaphore:
// a subtraction, undone for what was not there) and only then advances the
// head by what it got, so the head never passes the tail; an entry it takes
// may still be in the middle of its producer's write, which the flag tells.
// Reserve n entries; `room` = how many of them lie inside the pool (entries
// beyond its capacity are never written or taken).
__device__ __forceinline__ uint32_t pool_reserve(uint32_t* tail, uint32_t n, uint32_t cap,
                                                 uint32_t& room) {
  const uint32_t at = atomicAdd(tail, n);
  room = at >= cap ? 0u : min(n, cap - at);
  return at;
}
// Claim up to 32 published entries; returns how many and the first in h.
__device__ __forceinline__ uint32_t pool_take(uint32_t* head, int* avail, int want, uint32_t& h) {
  const int prev = atomicSub(avail, want);
  const int got = prev <= 0 ? 0 : min(prev, want);
  if (got < want) atomicAdd(avail, want - got);
  if (got > 0) h = atomicAdd(head, (uint32_t)got);
  return (uint32_t)got;
}

// Copy the first `room` of n (< 32) warp-queue entries to a drain pool at
// entry `at` (room == n), or publish `room` empty entries there when the
// pool ran out (room < n; the warp then traces all n itself); each lane one
// entry, published by its flag.
__device__ __forceinline__ void pool_put(const float4* q, float4* pool, uint32_t* flag,
                                         uint32_t at, uint32_t n, uint32_t room, uint32_t epoch) {
  const uint32_t lane = threadIdx.x & 31;
  if (lane < room) {
    float4* d = pool + 3 * ((size_t)at + lane);
    if (room == n) {
      const float4* e = q + 3 * (size_t)lane;
      const float4 e0 = e[0], e1 = e[1], e2 = e[2];
      d[0] = e0; d[1] = e1; d[2] = e2;
    } else {
      d[0] = make_float4(0.f, 0.f, 0.f, __uint_as_float(kNullPix));
    }
    st_release(flag + at + lane, epoch);
  }
}

__device__ __forceinline__ void flush_work(const WorkCount& wc, uint64_t* work, int kind) {
  uint32_t a = wc.inner, b = wc.sphere, c = wc.tri;
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xFFFFFFFFu, a, off);
    b += __shfl_down_sync(0xFFFFFFFFu, b, off);
    c += __shfl_down_sync(0xFFFFFFFFu, c, off);
  }
  if (lane_id() == 0) {
    atomicAdd((unsigned long long*)&work[3 * kind + 0], (unsigned long long)a);
    atomicAdd((unsigned long long*)&work[3 * kind + 1], (unsigned long long)b);
    atomicAdd((unsigned long long*)&work[3 * kind + 2], (unsigned long long)c);
  }
}

enum Mode : int { M_SHADOW = 0, M_PRIMARY = 1, M_MIRROR = 2 };

// Shadow queue entry: (origin | pixel) (direction | t_max) (contribution | 0)
// Mirror queue entry: (origin | pixel) (direction | depth) (weight | 0)
template <bool COUNT, int TREE>
__global__ void
#if RT_MIN_BLOCKS > 0
__launch_bounds__(kThreads, RT_MIN_BLOCKS)
#else
__launch_bounds__(kThreads)
#endif
k_render(KParams kp) {
  const RenderArgs& a = kp.a;
  // the top of the 4-wide tree, staged in shared memory once per block
  extern __shared__ float4 top[];
  if (TREE == kTreeWide4 && !COUNT) {
    for (uint32_t i = threadIdx.x; i < 7u * a.sc.n_top; i += blockDim.x) top[i] = a.sc.nodes4[i];
    __syncthreads();
  }
  const CameraParams& cam = a.cam;
  const uint32_t P = cam.W * cam.rows;   // pixels per eye of the traced rows, one frame
  // pixel ids: eye * FP + frame * P + row * W + column (eye-major: the left
  // eyes of all frames first, so each eye's sums and images are contiguous)
  const uint32_t FP = P * kp.n_frames;
  const uint32_t lane = lane_id();
  const uint32_t lt_mask = (1u << lane) - 1u;
  const size_t gwarp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  float4* const S = kp.wq + gwarp * 3 * (size_t)(kp.cap_s + kp.cap_r);
  float4* const R = S + 3 * (size_t)kp.cap_s;
  uint32_t* const cnt = kp.counters;
  uint32_t nS = 0, nR = 0;          // warp-uniform queue fills
  uint32_t made_s = 0, made_r = 0;  // rays this warp enqueued
  bool tiles_left = true;
  uint32_t tiles_out = 0;           // lane 0: the tiles-out flag, loaded one round ahead
  const uint32_t plist_n = a.plist_n_dev ? *a.plist_n_dev : a.plist_n;
  const uint32_t n_tiles = a.plist ? (plist_n + 31u) / 32u : kp.n_tiles;
  WorkCount wc_p = {0, 0, 0}, wc_s = {0, 0, 0}, wc_r = {0, 0, 0};
  const uint32_t L = a.sc.n_lights;

  for (uint32_t round = 0;; ++round) {
    if (round > (1u << 30)) { if (lane == 0) atomicOr(a.err, ERR_ITER); break; }
    // ---------------------------------------------- warp-uniform schedule
    int mode;
    uint32_t take = 0, tile = 0;
    const float4* src = nullptr;        // first queue entry of this round's batch
    const uint32_t* flags = nullptr;    // batch from a drain pool: its entries' flags
    // before a round on its own queue: have the tiles run out meanwhile?
    // then the queue goes to the pools instead (the flag was loaded during
    // the previous round, so its latency is hidden)
    if (tiles_left && (nS >= 32 || nR >= 32) && __shfl_sync(0xFFFFFFFFu, tiles_out, 0))
      tiles_left = false;
    if (tiles_left && nS >= 32) { mode = M_SHADOW; take = 32; nS -= 32; src = S + 3 * (size_t)nS; }
    else if (tiles_left && nR >= 32) { mode = M_MIRROR; take = 32; nR -= 32; src = R + 3 * (size_t)nR; }
    else if (tiles_left) {
      uint32_t t = 0;
      if (lane == 0) t = atomicAdd(&cnt[C_TILE], 1u);
      t = __shfl_sync(0xFFFFFFFFu, t, 0);
      if (t >= n_tiles) {
        if (lane == 0 && t == n_tiles) st_relaxed(&cnt[C_TILES_OUT], 1u);
        tiles_left = false;
        continue;
      }
      mode = M_PRIMARY; tile = t;
    } else {
      // ------------------------------------------------------ drain phase
      // hand the whole queue to the pools, 32 entries at a time, so that
      // every warp still running shares the rest of the frame
      bool keep_s = false, keep_r = false;   // a pool ran out: trace them here
      // in a small scene a backlog of less than a round per kind stays here:
      // its rounds cost less than handing them over (a few contended atomics
      // on the pool counters at the end of the frame)
      if (nS < 32 && nR < 32 && !kp.share_partial) { keep_s = nS > 0; keep_r = nR > 0; }
      else
      for (int kind = 0; kind < 2; ++kind) {
        uint32_t& nq = kind ? nR : nS;
        const size_t off = kind ? (size_t)kp.cap_p : 0;
        while (nq > 0) {
          const uint32_t c = min(nq, 32u);
          uint32_t at = 0, room = 0;
          if (lane == 0) {
            if (ld_relaxed(&cnt[kind ? C_R_TAIL : C_S_TAIL]) < kp.cap_p)
              at = pool_reserve(&cnt[kind ? C_R_TAIL : C_S_TAIL], c, kp.cap_p, room);
          }
          at = __shfl_sync(0xFFFFFFFFu, at, 0);
          room = __shfl_sync(0xFFFFFFFFu, room, 0);
          pool_put((kind ? R : S) + 3 * (size_t)(nq - c), kp.pool + 3 * off, kp.pool_flag + off,
                   at, c, room, kp.epoch);
          __syncwarp();
          if (lane == 0 && room > 0) atomicAdd((int*)&cnt[kind ? C_R_AVAIL : C_S_AVAIL], (int)room);
          if (room < c) { if (kind) keep_r = true; else keep_s = true; break; }
          nq -= c;
        }
      }
      if (keep_s) { mode = M_SHADOW; take = min(nS, 32u); nS -= take; src = S + 3 * (size_t)nS; }
      else if (keep_r) { mode = M_MIRROR; take = min(nR, 32u); nR -= take; src = R + 3 * (size_t)nR; }
      else {
        // take a batch, mirror rays first (they start the longest chains),
        // else shadow rays; nothing taken ends the warp (a lost race too:
        // retrying costs more in contention on the pool counters than the
        // warp adds, measured)
        uint32_t n = 0, h = 0, kind = 0;
        if (lane == 0) {
          const int2 av = ld_volatile2(&cnt[C_S_AVAIL]);   // (shadow, mirror) published
          if (av.y > 0) { n = pool_take(&cnt[C_R_HEAD], (int*)&cnt[C_R_AVAIL], 32, h); kind = 1; }
          if (n == 0 && av.x > 0) { n = pool_take(&cnt[C_S_HEAD], (int*)&cnt[C_S_AVAIL], 32, h); kind = 0; }
        }
        n = __shfl_sync(0xFFFFFFFFu, n, 0);
        h = __shfl_sync(0xFFFFFFFFu, h, 0);
        kind = __shfl_sync(0xFFFFFFFFu, kind, 0);
        if (n > 0) {
          const size_t off = kind ? (size_t)kp.cap_p : 0;
          mode = kind ? M_MIRROR : M_SHADOW;
          take = n;
          src = kp.pool + 3 * (off + h);
          flags = kp.pool_flag + off + h;
        } else {
          // nothing published in either pool: this warp is done. Every ray
          // handed to a pool is taken by a warp still running (at the latest
          // by the warp that handed it over, which looks again after handing
          // over), so no ray is left behind.
          break;
        }
      }
    }
    if (tiles_left && lane == 0) tiles_out = ld_relaxed(&cnt[C_TILES_OUT]);

    if (mode == M_SHADOW) {
      // ------------------------------------------------ any-hit round
      if (lane < take) {
        const float4* e = src + 3 * (size_t)lane;
        float4 s0, s1, s2;
        bool ok = true;
        if (flags) {                       // wait until the entry is published
          uint32_t spins = 0;
          while (ld_relaxed(flags + lane) != kp.epoch) {
            if (++spins > kSpinMax) { atomicOr(a.err, ERR_QUEUE); ok = false; break; }
            __nanosleep(64);
          }
          s0 = __ldcg(e); s1 = __ldcg(e + 1); s2 = __ldcg(e + 2);
        } else {
          s0 = e[0]; s1 = e[1]; s2 = e[2];
        }
        if (__float_as_uint(s0.w) >= 2 * FP) {    // an empty pool entry, or corrupt
          if (__float_as_uint(s0.w) != kNullPix) atomicOr(a.err, ERR_INDEX);
          ok = false;
        }
        float tb = 0.f;
        uint32_t id = 0, k = 0;
        if (ok && !trace_ray<true, COUNT, TREE>(a.sc, top, xyz(s0), xyz(s1), s1.w, tb, id, k, wc_s, a.err))
          accumulate(kp.accum, __float_as_uint(s0.w), s2.x, s2.y, s2.z, a.color_scale);
      }
      __syncwarp();
      continue;
    }

    // ------------------------------------------- closest hit + shading
    bool active;
    V3 o, d, w = v3(1.f, 1.f, 1.f);
    uint32_t pix = 0, depth = 0;
    if (mode == M_PRIMARY) {
      uint32_t eye, px, py, frame;
      if (a.plist) {                       // an explicit pixel list (masked retrace)
        const uint32_t i = tile * 32u + lane;
        active = i < plist_n;
        pix = active ? a.plist[i] : 0u;
        if (pix >= 2 * FP) { active = false; pix = 0u; }
        eye = pix >= FP;
        const uint32_t r = pix - eye * FP;
        frame = r / P;
        const uint32_t pi = r - frame * P;
        py = pi / cam.W;
        px = pi - py * cam.W;
      } else {
        frame = tile / kp.tiles_pf;
        const uint32_t ft = tile - frame * kp.tiles_pf;   // tile within its frame
        if (a.eyes == 3u && kp.pair_eyes) {   // 4x4 pixels of both eyes: lane 2q left, 2q+1 right
          const uint32_t tx4 = (cam.W + 3u) / 4u, q = lane >> 1;
          eye = lane & 1u;
          px = (ft % tx4) * 4u + (q & 3u);
          py = (ft / tx4) * 4u + (q >> 2);
        } else {                             // 8x4 tiles of one eye, eyes alternating when both are traced
          const uint32_t tt = a.eyes == 3u ? ft >> 1 : ft;
          eye = a.eyes == 3u ? (ft & 1u) : (a.eyes == 2u ? 1u : 0u);
          px = (tt % cam.tiles_x) * 8u + (lane & 7u);
          py = (tt / cam.tiles_x) * 4u + (lane >> 3);
        }
        active = px < cam.W && py < cam.rows;
        pix = eye * FP + frame * P + py * cam.W + px;
      }
      primary_ray(kp.cams[frame < kp.n_frames ? frame : 0], px, cam.y0 + py, eye, o, d);
    } else {
      active = lane < take;
      if (active) {
        const float4* e = src + 3 * (size_t)lane;
        float4 q0, q1, q2;
        if (flags) {                       // wait until the entry is published
          uint32_t spins = 0;
          while (ld_relaxed(flags + lane) != kp.epoch) {
            if (++spins > kSpinMax) { atomicOr(a.err, ERR_QUEUE); active = false; break; }
            __nanosleep(64);
          }
          q0 = __ldcg(e); q1 = __ldcg(e + 1); q2 = __ldcg(e + 2);
        } else {
          q0 = e[0]; q1 = e[1]; q2 = e[2];
        }
        o = xyz(q0);
        pix = __float_as_uint(q0.w);
        if (pix >= 2 * FP) {                        // an empty pool entry, or corrupt
          if (pix != kNullPix) atomicOr(a.err, ERR_INDEX);
          active = false;
          pix = 0;
        }
        d = xyz(q1);
        depth = __float_as_uint(q1.w);
        w = xyz(q2);
      }
      __syncwarp();  // every lane has read its entry before the slots are refilled
    }
    float t = INFINITY;
    uint32_t id = RT_MISS_ID, k = 0;
    bool hit = false;
    if (active)
      hit = trace_ray<false, COUNT, TREE>(a.sc, top, o, d, INFINITY, t, id, k,
                                   mode == M_PRIMARY ? wc_p : wc_r, a.err);
    __syncwarp();

    V3 p = v3(0.f, 0.f, 0.f), nrm = v3(0.f, 0.f, 1.f);
    float4 mat = make_float4(0.f, 0.f, 0.f, 0.f);
    float eps = 0.f;
    if (active) {
      float ar, ag, ab;
      if (!hit) {
        ar = w.x * kBgR; ag = w.y * kBgG; ab = w.z * kBgB;
      } else {
        hit_surface(a.sc.prims, a.sc.mats, a.sc.n_spheres, a.sc.n_mats, k, id, o, d, t, a.err, p,
                    nrm, mat, eps);
        const float kd = (1.f - mat.w) * kAmbient;
        ar = w.x * kd * mat.x; ag = w.y * kd * mat.y; ab = w.z * kd * mat.z;
      }
      if (RT_PRIMARY_STORE && mode == M_PRIMARY) store_first(kp.accum, pix, ar, ag, ab, a.color_scale);
      else accumulate(kp.accum, pix, ar, ag, ab, a.color_scale);
    }
    const bool lit = active && hit;
    const V3 o2 = p + nrm * eps;
    // shadow rays into this warp's queue, one per light facing the surface
    for (uint32_t l = 0; l < L; ++l) {
      bool emit = false;
      V3 lh = v3(0.f, 0.f, 1.f);
      float ld = 0.f, ndl = 0.f;
      if (lit) emit = light_ray(__ldg(a.sc.lights + l), o2, nrm, mat.w, lh, ld, ndl);
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, emit);
      const uint32_t slot = nS + __popc(m & lt_mask);
      if (emit && slot < kp.cap_s) {
        float4* e = S + 3 * (size_t)slot;
        e[0] = make_float4(o2.x, o2.y, o2.z, __uint_as_float(pix));
        e[1] = make_float4(lh.x, lh.y, lh.z, ld - eps);
        e[2] = make_float4(w.x * ndl * mat.x, w.y * ndl * mat.y, w.z * ndl * mat.z, 0.f);
      }
      nS += __popc(m);
      made_s += __popc(m);
    }
    // mirror ray into this warp's queue
    const bool refl = lit && mat.w > 0.f && depth < a.max_depth;
    const uint32_t mr = __ballot_sync(0xFFFFFFFFu, refl);
    const uint32_t rslot = nR + __popc(mr & lt_mask);
    if (refl && rslot < kp.cap_r) {
      const V3 rd = mirror_dir(d, nrm);
      float4* e = R + 3 * (size_t)rslot;
      e[0] = make_float4(o2.x, o2.y, o2.z, __uint_as_float(pix));
      e[1] = make_float4(rd.x, rd.y, rd.z, __uint_as_float(depth + 1));
      e[2] = make_float4(w.x * mat.w, w.y * mat.w, w.z * mat.w, 0.f);
    }
    nR += __popc(mr);
    made_r += __popc(mr);
    if (mode == M_PRIMARY && active) {
      const uint32_t eye = pix >= FP;
      const uint32_t pi = pix - eye * FP;  // frame * P + pixel
      uint32_t* hid = eye ? a.hit_R : a.hit_L;
      float* dep = eye ? a.depth_R : a.depth_L;
      if (hid) hid[pi] = id;
      if (dep) {
        const CameraParams& cf = kp.cams[pi / P];
        dep[pi] = hit ? t * dot(d, v3(cf.fwd[0], cf.fwd[1], cf.fwd[2])) : INFINITY;
      }
      if (!eye && a.refl_L) a.refl_L[pi] = hit ? mat.w : 0.f;
      float* nr = eye ? a.normal_R : a.normal_L;
      if (nr) {                            // zero normal on a miss
        nr[3 * (size_t)pi + 0] = hit ? nrm.x : 0.f;
        nr[3 * (size_t)pi + 1] = hit ? nrm.y : 0.f;
        nr[3 * (size_t)pi + 2] = hit ? nrm.z : 0.f;
      }
    }
    if (nS > kp.cap_s || nR > kp.cap_r) {  // cannot happen by construction; writes were skipped
      if (lane == 0) atomicOr(a.err, ERR_QUEUE);
      break;
    }
    __syncwarp();
  }
  if (lane == 0) {
    atomicAdd(&kp.counters[C_SHADOW], made_s);
    atomicAdd(&kp.counters[C_REFL], made_r);
  }
  if (COUNT) {
    flush_work(wc_p, a.work, 0);
    flush_work(wc_s, a.work, 1);
    flush_work(wc_r, a.work, 2);
  }
}

__global__ void k_resolve(const uint32_t* __restrict__ acc, float* __restrict__ out_L,
                          float* __restrict__ out_R, uint32_t n3, float inv_scale) {
  const uint32_t total = out_R ? 2 * n3 : n3;      // no right image: the left eye only
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const float v = fminf(1.f, (float)acc[i] * inv_scale);
    if (i < n3) out_L[i] = v; else out_R[i - n3] = v;
  }
}

// The same, 4 values per thread with 16-byte loads and stores, when n3 is a
// multiple of 4 and both images are 16-byte aligned: the images may be
// pinned host memory mapped into the device (the host-output render), where
// wide stores make fuller transfers over the CPU-GPU link.
__global__ void k_resolve4(const uint4* __restrict__ acc, float4* __restrict__ out_L,
                           float4* __restrict__ out_R, uint32_t n3_4, float inv_scale) {
  const uint32_t total = out_R ? 2 * n3_4 : n3_4;  // no right image: the left eye only
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const uint4 a = acc[i];
    const float4 v = make_float4(fminf(1.f, (float)a.x * inv_scale), fminf(1.f, (float)a.y * inv_scale),
                                 fminf(1.f, (float)a.z * inv_scale), fminf(1.f, (float)a.w * inv_scale));
    if (i < n3_4) out_L[i] = v; else out_R[i - n3_4] = v;
  }
}

__global__ void k_counts(const uint32_t* counters, uint64_t primary, uint64_t* out) {
  if (threadIdx.x != 0) return;
  out[0] = primary;
  out[1] = counters[C_SHADOW];
  out[2] = counters[C_REFL];
}

template <bool COUNT, int TREE>
int blocks_per_sm() {
  static int cached = 0;
  if (!cached) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render<COUNT, TREE>, kThreads,
                                                  kMaxTopBytes);
    cached = per_sm > 0 ? per_sm : 1;
  }
  return cached;
}

template <bool COUNT, int TREE>
cudaError_t render_impl(const RenderArgs& a, Workspace& ws, cudaStream_t st) {
  const uint32_t F = a.n_frames ? a.n_frames : 1u;
  if (F > (uint32_t)kMaxFrames) return cudaErrorInvalidValue;
  const uint64_t P = (uint64_t)a.cam.W * a.cam.rows * F;   // pixels per eye over all frames
  KParams kp;
  kp.a = a;
  kp.n_frames = F;
  for (uint32_t f = 0; f < F; ++f) kp.cams[f] = a.frames ? a.frames[f] : a.cam;
  kp.accum = ws.accum;
  kp.wq = ws.wq;
  kp.counters = ws.counters;
  kp.cap_s = ws.cap_s;
  kp.cap_r = ws.cap_r;
  kp.pair_eyes = a.eyes == 3u && a.sc.n_prims >= kPairEyesPrims;
  kp.tiles_pf = kp.pair_eyes ? ((a.cam.W + 3u) / 4u) * a.cam.tiles_y   // 4x4 pixels, both eyes
                             : (a.eyes == 3u ? 2u : 1u) * a.cam.tiles_x * a.cam.tiles_y;   // 8x4, one eye
  kp.n_tiles = a.plist ? (a.plist_n + 31u) / 32u : F * kp.tiles_pf;
  const int grid = render_grid();
  if ((uint64_t)grid * (kThreads / 32) > ws.n_warps) return cudaErrorInvalidValue;
  kp.share_partial = a.sc.n_prims >= kSharePartialPrims;
  kp.pool = ws.pool;
  kp.pool_flag = ws.pool_flag;
  kp.cap_p = ws.cap_p_limit && ws.cap_p_limit < ws.cap_p ? ws.cap_p_limit : ws.cap_p;
  if (++ws.epoch == 0) {            // flags of 2^32 renders ago could match: clear them
    cudaMemsetAsync(ws.pool_flag, 0, 2 * (size_t)ws.cap_p * sizeof(uint32_t), st);
    ws.epoch = 1;
  }
  kp.epoch = ws.epoch;
  cudaMemsetAsync(ws.counters, 0, C_TOTAL * sizeof(uint32_t), st);
  // the colour sums of the traced pixels start at their primary ray's store;
  // with atomic adds only, clear the sums of the eyes this render traces
  if (!RT_PRIMARY_STORE) {
    const bool left = !a.plist && (a.eyes & 1u), right = a.plist || (a.eyes & 2u);
    if (left && right) cudaMemsetAsync(ws.accum, 0, 2 * P * 3 * sizeof(uint32_t), st);
    else if (left) cudaMemsetAsync(ws.accum, 0, P * 3 * sizeof(uint32_t), st);
    else cudaMemsetAsync(ws.accum + 3 * P, 0, P * 3 * sizeof(uint32_t), st);
  }
  if (a.work) cudaMemsetAsync(a.work, 0, 9 * sizeof(uint64_t), st);
  profile_mark(ws, ST_CLEAR, st);
  const size_t top_bytes = (TREE == kTreeWide4 && !COUNT) ? 7 * sizeof(float4) * a.sc.n_top : 0;
  k_render<COUNT, TREE><<<grid, kThreads, top_bytes, st>>>(kp);
  profile_mark(ws, a.trace_stage, st);
  const uint32_t n3 = (uint32_t)(P * 3);
  if (a.resolve) {
    const bool wide = n3 % 4 == 0 && ((uintptr_t)a.out_L % 16) == 0 && ((uintptr_t)a.out_R % 16) == 0;
    if (wide)
      k_resolve4<<<num_sms() * 8, 256, 0, st>>>(reinterpret_cast<const uint4*>(ws.accum),
                                                 reinterpret_cast<float4*>(a.out_L),
                                                 reinterpret_cast<float4*>(a.out_R), n3 / 4,
                                                 1.f / a.color_scale);
    else
      k_resolve<<<num_sms() * 8, 256, 0, st>>>(ws.accum, a.out_L, a.out_R, n3, 1.f / a.color_scale);
    profile_mark(ws, ST_RESOLVE, st);
  }
  const uint64_t primary = a.plist ? a.plist_n : (a.eyes == 3u ? 2 * P : P);
  if (a.ray_counts && !a.plist_n_dev) k_counts<<<1, 32, 0, st>>>(ws.counters, primary, a.ray_counts);
  return cudaGetLastError();
}

}  // namespace

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

int render_grid() {
  // the variants may fit different numbers of blocks; size for the largest grid
  int b = blocks_per_sm<false, kTreeWide4>();
  if (blocks_per_sm<false, kTreeBinary>() > b) b = blocks_per_sm<false, kTreeBinary>();
  if (blocks_per_sm<true, kTreeBinary>() > b) b = blocks_per_sm<true, kTreeBinary>();
  return num_sms() * b;
}

int render_threads() { return kThreads; }

int treelet_depth() { return RT_TREELET_DEPTH; }

void profile_begin(Workspace& ws, cudaStream_t st) {
  ws.n_ev = 0;
  if (!ws.profile) return;
  ws.ev_stage[0] = -1;
  cudaEventRecord(ws.ev[ws.n_ev++], st);
}

void profile_mark(Workspace& ws, int stage, cudaStream_t st) {
  if (!ws.profile || ws.n_ev >= kMaxEvents) return;
  ws.ev_stage[ws.n_ev] = stage;
  cudaEventRecord(ws.ev[ws.n_ev++], st);
}

cudaError_t render(const RenderArgs& a, Workspace& ws, cudaStream_t st) {
  if (a.sc.n_top * 7 * sizeof(float4) > (size_t)kMaxTopBytes) return cudaErrorInvalidValue;
  if (a.work) return render_impl<true, kTreeBinary>(a, ws, st);
  if (a.tree == kTreeWide4 && a.sc.n4 > 0) return render_impl<false, kTreeWide4>(a, ws, st);
  return render_impl<false, kTreeBinary>(a, ws, st);
}

}  // namespace rt
