// Batched stereo rendering (sm_103a): many stereo requests of uneven
// resolutions, reflection depths and scenes in ONE persistent launch,
// replayed from a captured CUDA graph, with a measured autotuner for the
// launch shape.
//
// Paper Sec. 3 / Figure 1: the image is split into parts traced by parallel
// workers; here the parts of every request of a batch form one work list.
// Tiles of 32 rays are numbered request after request in the chosen order:
// tile_w x tile_h = 16 pixels traced for both eyes, the two rays of a pixel in
// neighbouring lanes (as the single-pair renderer does), or 32 pixels of one
// eye, the two eyes of a request alternating between tiles; warps pull tiles
// from one global counter, so small and large requests share the GPU without
// a launch per request or per bounce depth. Each warp keeps the single-pair
// renderer's two private wavefront queues (shadow rays, mirror rays); an
// entry now also carries its request, because a warp's queue may hold the
// tail of one request's tile next to the next request's rays. Traversal and
// shading use the same device functions as the single-pair renderer, and the
// colour sums are the same fixed-point integers, so every request's images
// equal rt_render_stereo's bit for bit, whatever the tile shape, order or
// residency.
//
// Paper Sec. 4 / Figure 8 measures the effect of the CUDA launch shape; the
// autotuner makes that choice per batch by timing candidates (coordinate
// descent over tile shape, blocks per SM, mirror-queue capacity and request
// order) with CUDA events.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "rt_internal.cuh"
#include "trace_dev.cuh"

namespace rt {
namespace {

// one request as the kernels see it (launch order)
struct BatchReq {
  CameraParams cam;        // tiles_x / tiles_y for the batch's tile shape
  DeviceScene sc;
  float color_scale;       // fixed-point scale of the scene's colour sums
  float inv_scale;         // 1 / color_scale (host division, as the single-pair resolve)
  uint32_t max_depth;
  uint32_t pix_base;       // global pixel id of (left eye, pixel 0); right eye follows at + W*H
  uint32_t tile_base;      // first tile in the work list
  uint32_t n_tiles;        // tiles_x * tiles_y (both eyes per tile), else twice that
  uint32_t user;           // index in the caller's request array
  uint32_t pad;
  float* out_L;
  float* out_R;
};

struct KBatch {
  const BatchReq* __restrict__ req;
  uint32_t n_req;
  uint32_t n_tiles;
  uint32_t tw_log2;        // tile width = 1 << tw_log2
  uint32_t paired;         // 1: 16-pixel tiles of both eyes (height 16 >> tw_log2), 0: 32 of one
  uint32_t cap_s, cap_r, q_stride;   // queue capacities and per-warp stride in entries
  uint32_t* accum;
  float4* wq;
  uint32_t* counters;
  uint32_t* err;
  unsigned long long* done_ns;       // per launch-order request, nullable
};

constexpr uint32_t kNoReq = 0xFFFFFFFFu;

// minimum resident blocks per SM requested from the register allocator for
// k_render_batch (9: 56 registers, no spills; the 64 requests of the batch
// workload take 57.9 ms against 59.7 at 8 blocks and 58.2 at 10)
#ifndef RT_BATCH_MIN_BLOCKS
#define RT_BATCH_MIN_BLOCKS 9
#endif

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ DeviceScene traversal_scene(const BatchReq* rq) {
  DeviceScene s = {};
  s.nodes = rq->sc.nodes;
  s.prims = rq->sc.prims;
  s.n_prims = rq->sc.n_prims;
  s.n_spheres = rq->sc.n_spheres;
  return s;
}

// the request owning tile t: warp-uniform binary search over tile_base
__device__ __forceinline__ uint32_t find_request(const KBatch& kp, uint32_t t, uint32_t hint) {
  if (hint < kp.n_req) {
    const uint32_t b = kp.req[hint].tile_base;
    if (t >= b && t - b < kp.req[hint].n_tiles) return hint;
  }
  uint32_t lo = 0, hi = kp.n_req - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (kp.req[mid].tile_base <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// stamp the requests this warp just worked on (one atomic per distinct request)
__device__ __forceinline__ void stamp(const KBatch& kp, uint32_t r) {
  const uint32_t act = __ballot_sync(0xFFFFFFFFu, r != kNoReq);
  if (r == kNoReq) return;
  const uint32_t grp = __match_any_sync(act, r);
  if (lane_id() == (uint32_t)(__ffs(grp) - 1)) atomicMax(kp.done_ns + r, global_ns());
}

__global__ void k_stamp(unsigned long long* t) {
  if (threadIdx.x == 0) *t = global_ns();
}

// Shadow queue entry: (origin | pixel) (direction | t_max) (contribution | request)
// Mirror queue entry: (origin | pixel) (direction | depth) (weight | request)
__global__ void __launch_bounds__(kThreads, RT_BATCH_MIN_BLOCKS) k_render_batch(KBatch kp) {
  const uint32_t lane = lane_id();
  const uint32_t lt_mask = (1u << lane) - 1u;
  const size_t gwarp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  float4* const S = kp.wq + gwarp * 3 * (size_t)kp.q_stride;
  float4* const R = S + 3 * (size_t)kp.cap_s;
  const uint32_t tw_mask = (1u << kp.tw_log2) - 1u;
  uint32_t nS = 0, nR = 0;
  uint32_t made_s = 0, made_r = 0;
  bool tiles_left = true;
  uint32_t hint = kNoReq;
  WorkCount wc = {0, 0, 0};

  for (uint32_t round = 0;; ++round) {
    if (round > (1u << 30)) { if (lane == 0) atomicOr(kp.err, ERR_ITER); break; }
    int mode;
    uint32_t take = 0, base = 0, tile = 0;
    if (nS >= 32) { mode = 0; take = 32; nS -= 32; base = nS; }
    else if (nR >= 32) { mode = 2; take = 32; nR -= 32; base = nR; }
    else if (tiles_left) {
      uint32_t t = 0;
      if (lane == 0) t = atomicAdd(&kp.counters[C_TILE], 1u);
      t = __shfl_sync(0xFFFFFFFFu, t, 0);
      if (t >= kp.n_tiles) { tiles_left = false; continue; }
      mode = 1; tile = t;
    }
    else if (nS > 0) { mode = 0; take = nS; base = 0; nS = 0; }
    else if (nR > 0) { mode = 2; take = nR; base = 0; nR = 0; }
    else break;

    if (mode == 0) {
      // ------------------------------------------------ any-hit round
      uint32_t r = kNoReq;
      if (lane < take) {
        const float4* e = S + 3 * (size_t)(base + lane);
        const float4 s0 = e[0], s1 = e[1], s2 = e[2];
        r = __float_as_uint(s2.w);
        if (r < kp.n_req) {
          const BatchReq* rq = kp.req + r;
          float tb = 0.f;
          uint32_t id = 0, k = 0;
          const bool blocked = traverse<true, false>(traversal_scene(rq), xyz(s0), xyz(s1), s1.w,
                                                     tb, id, k, wc, kp.err);
          if (!blocked) accumulate(kp.accum, __float_as_uint(s0.w), s2.x, s2.y, s2.z, rq->color_scale);
        } else {
          atomicOr(kp.err, ERR_INDEX);
          r = kNoReq;
        }
      }
      if (kp.done_ns) stamp(kp, r);
      __syncwarp();
      continue;
    }

    // ------------------------------------------- closest hit + shading
    bool active;
    V3 o = v3(0.f, 0.f, 0.f), d = v3(0.f, 0.f, 1.f), w = v3(1.f, 1.f, 1.f);
    uint32_t pix = 0, depth = 0, r = kNoReq;
    if (mode == 1) {
      r = find_request(kp, tile, hint);
      hint = r;
      const BatchReq* rq = kp.req + r;
      const uint32_t lt = tile - rq->tile_base;
      const uint32_t eye = kp.paired ? lane & 1u : lt & 1u;
      const uint32_t tt = kp.paired ? lt : lt >> 1, q = kp.paired ? lane >> 1 : lane;
      const uint32_t W = rq->cam.W, H = rq->cam.H, tx = rq->cam.tiles_x;
      const uint32_t px = (tt % tx) * (tw_mask + 1u) + (q & tw_mask);
      const uint32_t py = (tt / tx) * ((kp.paired ? 16u : 32u) >> kp.tw_log2) + (q >> kp.tw_log2);
      active = px < W && py < H;
      pix = rq->pix_base + eye * (W * H) + py * W + px;
      if (active) primary_ray(rq->cam, px, py, eye, o, d);
      if (!active) r = kNoReq;
    } else {
      active = lane < take;
      if (active) {
        const float4* e = R + 3 * (size_t)(base + lane);
        const float4 q0 = e[0], q1 = e[1], q2 = e[2];
        o = xyz(q0);
        pix = __float_as_uint(q0.w);
        d = xyz(q1);
        depth = __float_as_uint(q1.w);
        w = xyz(q2);
        r = __float_as_uint(q2.w);
        if (r >= kp.n_req) { atomicOr(kp.err, ERR_INDEX); active = false; r = kNoReq; }
      }
      __syncwarp();  // every lane has read its entry before the slots are refilled
    }
    const BatchReq* rq = kp.req + (active ? r : 0u);
    float t = INFINITY;
    uint32_t id = RT_MISS_ID, k = 0;
    bool hit = false;
    if (active) hit = traverse<false, false>(traversal_scene(rq), o, d, INFINITY, t, id, k, wc, kp.err);
    __syncwarp();

    V3 p = v3(0.f, 0.f, 0.f), nrm = v3(0.f, 0.f, 1.f);
    float4 mat = make_float4(0.f, 0.f, 0.f, 0.f);
    float eps = 0.f, scale = 0.f;
    uint32_t L = 0, max_depth = 0;
    const float4* lights = nullptr;
    if (active) {
      scale = rq->color_scale;
      float ar, ag, ab;
      if (!hit) {
        ar = w.x * kBgR; ag = w.y * kBgG; ab = w.z * kBgB;
      } else {
        hit_surface(rq->sc.prims, rq->sc.mats, rq->sc.n_spheres, rq->sc.n_mats, k, id, o, d, t,
                    kp.err, p, nrm, mat, eps);
        const float kd = (1.f - mat.w) * kAmbient;
        ar = w.x * kd * mat.x; ag = w.y * kd * mat.y; ab = w.z * kd * mat.z;
        L = rq->sc.n_lights;
        lights = rq->sc.lights;
        max_depth = rq->max_depth;
      }
      if (RT_PRIMARY_STORE && mode == 1) store_first(kp.accum, pix, ar, ag, ab, scale);
      else accumulate(kp.accum, pix, ar, ag, ab, scale);
    }
    const bool lit = active && hit;
    const V3 o2 = p + nrm * eps;
    const uint32_t Lmax = __reduce_max_sync(0xFFFFFFFFu, L);
    for (uint32_t l = 0; l < Lmax; ++l) {
      bool emit = false;
      V3 lh = v3(0.f, 0.f, 1.f);
      float ld = 0.f, ndl = 0.f;
      if (lit && l < L) emit = light_ray(__ldg(lights + l), o2, nrm, mat.w, lh, ld, ndl);
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, emit);
      const uint32_t slot = nS + __popc(m & lt_mask);
      if (emit && slot < kp.cap_s) {
        float4* e = S + 3 * (size_t)slot;
        e[0] = make_float4(o2.x, o2.y, o2.z, __uint_as_float(pix));
        e[1] = make_float4(lh.x, lh.y, lh.z, ld - eps);
        e[2] = make_float4(w.x * ndl * mat.x, w.y * ndl * mat.y, w.z * ndl * mat.z,
                           __uint_as_float(r));
      }
      nS += __popc(m);
      made_s += __popc(m);
    }
    const bool refl = lit && mat.w > 0.f && depth < max_depth;
    const uint32_t mr = __ballot_sync(0xFFFFFFFFu, refl);
    const uint32_t rslot = nR + __popc(mr & lt_mask);
    if (refl && rslot < kp.cap_r) {
      const V3 rd = mirror_dir(d, nrm);
      float4* e = R + 3 * (size_t)rslot;
      e[0] = make_float4(o2.x, o2.y, o2.z, __uint_as_float(pix));
      e[1] = make_float4(rd.x, rd.y, rd.z, __uint_as_float(depth + 1));
      e[2] = make_float4(w.x * mat.w, w.y * mat.w, w.z * mat.w, __uint_as_float(r));
    }
    nR += __popc(mr);
    made_r += __popc(mr);
    if (kp.done_ns) stamp(kp, active ? r : kNoReq);
    if (nS > kp.cap_s || nR > kp.cap_r) {  // cannot happen by construction; writes were skipped
      if (lane == 0) atomicOr(kp.err, ERR_QUEUE);
      break;
    }
    __syncwarp();
  }
  if (lane == 0) {
    atomicAdd(&kp.counters[C_SHADOW], made_s);
    atomicAdd(&kp.counters[C_REFL], made_r);
  }
}

// fixed-point sums -> float RGB; blockIdx.y = request (launch order)
__global__ void k_resolve_batch(const BatchReq* __restrict__ req, const uint32_t* __restrict__ acc) {
  const BatchReq& rq = req[blockIdx.y];
  const uint32_t n3 = 3u * rq.cam.W * rq.cam.H;
  const uint32_t* a = acc + 3 * (size_t)rq.pix_base;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * n3; i += gridDim.x * blockDim.x) {
    const float v = fminf(1.f, (float)a[i] * rq.inv_scale);
    if (i < n3) rq.out_L[i] = v; else rq.out_R[i - n3] = v;
  }
}

int batch_occupancy() {
  static int cached = 0;
  if (!cached) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_batch, kThreads, 0);
    cached = per_sm > 0 ? per_sm : 1;
  }
  return cached;
}

constexpr uint32_t kCapRMax = 256;

bool valid_config(const rt_batch_config& c) {
  const bool tile = (c.tile_w == 4 && c.tile_h == 8) || (c.tile_w == 8 && c.tile_h == 4) ||
                    (c.tile_w == 16 && c.tile_h == 2) || (c.tile_w == 32 && c.tile_h == 1) ||
                    (c.tile_w == 2 && c.tile_h == 8) || (c.tile_w == 4 && c.tile_h == 4) ||
                    (c.tile_w == 8 && c.tile_h == 2) || (c.tile_w == 16 && c.tile_h == 1);
  const bool cap = c.cap_r == 64 || c.cap_r == 128 || c.cap_r == 256;
  return tile && cap && c.order <= RT_BATCH_ORDER_SMALLEST_FIRST && c.track_latency <= 1 &&
         (int)c.blocks_per_sm <= batch_occupancy();
}

}  // namespace
}  // namespace rt

// the opaque batch of the C-ABI
struct rt_batch {
  int device = 0;
  std::vector<rt_request> reqs;          // caller order
  std::vector<rt::RenderArgs> args;      // validated arguments per request (caller order)
  std::vector<uint32_t> pix_base;        // caller order
  std::vector<uint32_t> pos;             // caller index -> launch-order position
  rt_batch_config cfg = {};
  uint32_t n = 0, n_tiles = 0, max_lights = 0;
  uint64_t total_pixels = 0;
  uint64_t primary_rays = 0;
  rt::BatchReq* h_table = nullptr;       // pinned, launch order
  rt::BatchReq* d_table = nullptr;
  void* block = nullptr;
  uint32_t* accum = nullptr;
  float4* wq = nullptr;
  uint32_t* counters = nullptr;
  uint32_t* err = nullptr;
  unsigned long long* done_ns = nullptr;  // n + 1: per request, then the start stamp
  uint32_t cap_s = 0, q_stride = 0;
  uint64_t n_warps = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t last = nullptr;
  bool launched = false;
};

using rt::cuda_fail;
using rt::fail;

static_assert(sizeof(rt_request) == 88 && offsetof(rt_request, camera) == 8 &&
                  offsetof(rt_request, eye_sep) == 48 && offsetof(rt_request, W) == 56 &&
                  offsetof(rt_request, reserved) == 68 && offsetof(rt_request, d_out_L) == 72,
              "rt_request layout");
static_assert(sizeof(rt_batch_config) == 24, "rt_batch_config layout");

namespace {

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

void drop_graph(rt_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// launch-order table and graph for configuration c
int apply_config(rt_batch* b, const rt_batch_config& c) {
  if (b->launched) cudaEventSynchronize(b->last);
  const uint32_t tw = c.tile_w, th = c.tile_h;
  uint32_t tw_log2 = 0;
  while ((1u << tw_log2) < tw) ++tw_log2;
  std::vector<uint32_t> order(b->n);
  std::iota(order.begin(), order.end(), 0u);
  auto px = [&](uint32_t i) { return (uint64_t)b->reqs[i].W * b->reqs[i].H; };
  if (c.order == RT_BATCH_ORDER_LARGEST_FIRST)
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return px(x) > px(y); });
  else if (c.order == RT_BATCH_ORDER_SMALLEST_FIRST)
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return px(x) < px(y); });
  uint64_t tiles = 0;
  for (uint32_t j = 0; j < b->n; ++j) {
    const uint32_t i = order[j];
    const rt::RenderArgs& a = b->args[i];
    rt::BatchReq& q = b->h_table[j];
    std::memset(&q, 0, sizeof q);
    q.cam = a.cam;
    q.cam.tiles_x = (a.cam.W + tw - 1) / tw;
    q.cam.tiles_y = (a.cam.H + th - 1) / th;
    q.sc = a.sc;
    q.color_scale = a.color_scale;
    q.inv_scale = 1.f / a.color_scale;
    q.max_depth = a.max_depth;
    q.pix_base = b->pix_base[i];
    q.tile_base = (uint32_t)tiles;
    q.n_tiles = (tw * th == 16 ? 1u : 2u) * q.cam.tiles_x * q.cam.tiles_y;
    q.user = i;
    q.out_L = b->reqs[i].d_out_L;
    q.out_R = b->reqs[i].d_out_R;
    tiles += q.n_tiles;
    b->pos[i] = j;
  }
  if (tiles >= (1ull << 32)) return fail(RT_ERR_INVALID_ARG, "batch has 2^32 or more tiles");
  b->n_tiles = (uint32_t)tiles;
  const int bps = c.blocks_per_sm ? (int)c.blocks_per_sm : rt::batch_occupancy();
  const int grid = rt::num_sms() * bps;
  if ((uint64_t)grid * (rt::kThreads / 32) > b->n_warps) return fail(RT_ERR_INVALID_ARG, "grid exceeds the queue allocation");

  rt::KBatch kp;
  kp.req = b->d_table;
  kp.n_req = b->n;
  kp.n_tiles = b->n_tiles;
  kp.tw_log2 = tw_log2;
  kp.paired = tw * th == 16 ? 1u : 0u;
  kp.cap_s = b->cap_s;
  kp.cap_r = c.cap_r;
  kp.q_stride = b->q_stride;
  kp.accum = b->accum;
  kp.wq = b->wq;
  kp.counters = b->counters;
  kp.err = b->err;
  kp.done_ns = c.track_latency ? b->done_ns : nullptr;

  drop_graph(b);
  cudaStream_t st = b->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "rt_batch: begin capture");
  cudaMemcpyAsync(b->d_table, b->h_table, sizeof(rt::BatchReq) * b->n, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(b->counters, 0, rt::C_TOTAL * sizeof(uint32_t), st);
  cudaMemsetAsync(b->err, 0, sizeof(uint32_t), st);
  if (!RT_PRIMARY_STORE) cudaMemsetAsync(b->accum, 0, b->total_pixels * 3 * sizeof(uint32_t), st);
  if (c.track_latency) {
    cudaMemsetAsync(b->done_ns, 0, (size_t)b->n * sizeof(unsigned long long), st);
    rt::k_stamp<<<1, 32, 0, st>>>(b->done_ns + b->n);
  }
  rt::k_render_batch<<<grid, rt::kThreads, 0, st>>>(kp);
  rt::k_resolve_batch<<<dim3(rt::num_sms() * 2, b->n), 256, 0, st>>>(b->d_table, b->accum);
  const cudaError_t launch_err = cudaGetLastError();
  e = cudaStreamEndCapture(st, &b->graph);
  if (launch_err != cudaSuccess) { drop_graph(b); return cuda_fail(launch_err, "rt_batch: capture"); }
  if (e != cudaSuccess) { cudaGetLastError(); drop_graph(b); return cuda_fail(e, "rt_batch: end capture"); }
  e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) { cudaGetLastError(); drop_graph(b); return cuda_fail(e, "rt_batch: instantiate"); }
  b->cfg = c;
  b->cfg.blocks_per_sm = (uint32_t)bps;
  return RT_OK;
}

void free_batch(rt_batch* b) {
  if (b->launched && b->last) cudaEventSynchronize(b->last);
  drop_graph(b);
  if (b->last) cudaEventDestroy(b->last);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->block) cudaFree(b->block);
  if (b->d_table) cudaFree(b->d_table);
  if (b->h_table) cudaFreeHost(b->h_table);
  delete b;
}

int check_status(rt_batch* b) {
  uint32_t h = 0;
  const cudaError_t e = cudaMemcpy(&h, b->err, sizeof h, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "rt_batch: status read");
  if (h & rt::ERR_ITER) return fail(RT_ERR_TIMEOUT, "batched render: a traversal or scheduling loop hit its iteration bound");
  if (h) return fail(RT_ERR_DEVICE_CHECK, "batched render: device-side check failed (flags " + std::to_string(h) + ")");
  return RT_OK;
}

}  // namespace

extern "C" {

int rt_batch_create(const rt_request* reqs, uint32_t n_requests, const rt_batch_config* cfg,
                    rt_batch** out_batch) {
  if (!out_batch) return fail(RT_ERR_INVALID_ARG, "out_batch is NULL");
  *out_batch = nullptr;
  if (!reqs) return fail(RT_ERR_INVALID_ARG, "reqs is NULL");
  if (n_requests < 1 || n_requests > RT_BATCH_MAX_REQUESTS)
    return fail(RT_ERR_INVALID_ARG, "n_requests must be in 1..RT_BATCH_MAX_REQUESTS");
  rt_batch_config c = {4, 4, 0, 64, RT_BATCH_ORDER_LARGEST_FIRST, 1};
  if (cfg) c = *cfg;
  for (uint32_t i = 0; i < n_requests; ++i) {
    const rt_request& r = reqs[i];
    if (!r.scene) return fail(RT_ERR_INVALID_ARG, "request " + std::to_string(i) + ": scene is NULL");
    if (!r.d_out_L || !r.d_out_R) return fail(RT_ERR_INVALID_ARG, "request " + std::to_string(i) + ": output is NULL");
    if (r.reserved) return fail(RT_ERR_INVALID_ARG, "request " + std::to_string(i) + ": reserved must be 0");
  }
  rt_batch* b = new (std::nothrow) rt_batch();
  if (!b) return fail(RT_ERR_OOM, "rt_batch_create: host allocation");
  b->n = n_requests;
  b->reqs.assign(reqs, reqs + n_requests);
  b->args.resize(n_requests);
  b->pix_base.resize(n_requests);
  b->pos.resize(n_requests);
  uint64_t pixels = 0;
  for (uint32_t i = 0; i < n_requests; ++i) {
    const rt_request& r = reqs[i];
    const int rc = rt::make_render_args(r.scene, &r.camera, r.eye_sep, r.convergence, r.W, r.H,
                                        r.max_depth, b->args[i]);
    if (rc != RT_OK) { delete b; return rc; }
    b->pix_base[i] = (uint32_t)pixels;
    pixels += 2ull * r.W * r.H;
    if (pixels >= (1ull << 32)) { delete b; return fail(RT_ERR_INVALID_ARG, "sum of 2*W*H must stay below 2^32"); }
    b->max_lights = std::max(b->max_lights, b->args[i].sc.n_lights);
  }
  b->total_pixels = pixels;
  b->primary_rays = pixels;
  cudaGetDevice(&b->device);
  if (!rt::valid_config(c)) {
    delete b;
    return fail(RT_ERR_INVALID_ARG, "rt_batch_config: unsupported tile shape, cap_r, order or blocks_per_sm");
  }
  // device memory: colour sums, per-warp queues (sized for the largest
  // candidate grid and mirror queue), counters, error word, timestamps
  b->cap_s = 32u * b->max_lights + 32u;
  b->q_stride = b->cap_s + rt::kCapRMax;
  b->n_warps = (uint64_t)rt::num_sms() * rt::batch_occupancy() * (rt::kThreads / 32);
  const size_t b_acc = align256(pixels * 3 * sizeof(uint32_t));
  const size_t b_q = align256(b->n_warps * b->q_stride * 3 * sizeof(float4));
  const size_t b_c = align256(rt::C_TOTAL * sizeof(uint32_t) + sizeof(uint32_t));
  const size_t b_t = align256((size_t)(n_requests + 1) * sizeof(unsigned long long));
  cudaError_t e = cudaMalloc(&b->block, b_acc + b_q + b_c + b_t);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->d_table), sizeof(rt::BatchReq) * n_requests);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&b->h_table), sizeof(rt::BatchReq) * n_requests);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->last, cudaEventDisableTiming);
  if (e != cudaSuccess) { cudaGetLastError(); free_batch(b); return cuda_fail(e, "rt_batch_create: allocation"); }
  char* p = static_cast<char*>(b->block);
  b->accum = reinterpret_cast<uint32_t*>(p); p += b_acc;
  b->wq = reinterpret_cast<float4*>(p); p += b_q;
  b->counters = reinterpret_cast<uint32_t*>(p);
  b->err = b->counters + rt::C_TOTAL;
  p += b_c;
  b->done_ns = reinterpret_cast<unsigned long long*>(p);
  const int rc = apply_config(b, c);
  if (rc != RT_OK) { free_batch(b); return rc; }
  *out_batch = b;
  return RT_OK;
}

void rt_batch_destroy(rt_batch* batch) {
  if (batch) free_batch(batch);
}

int rt_batch_launch(rt_batch* batch, void* cuda_stream) {
  if (!batch || !batch->exec) return fail(RT_ERR_INVALID_ARG, "batch is NULL or has no graph");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGraphLaunch(batch->exec, st);
  if (e == cudaSuccess) e = cudaEventRecord(batch->last, st);
  if (e != cudaSuccess) return cuda_fail(e, "rt_batch_launch");
  batch->launched = true;
  return RT_OK;
}

int rt_batch_set_camera(rt_batch* batch, uint32_t i, const rt_camera* cam, float eye_sep,
                        float convergence) {
  if (!batch || i >= batch->n) return fail(RT_ERR_INVALID_ARG, "batch is NULL or index out of range");
  rt_request r = batch->reqs[i];
  rt::RenderArgs a;
  const int rc = rt::make_render_args(r.scene, cam, eye_sep, convergence, r.W, r.H, r.max_depth, a);
  if (rc != RT_OK) return rc;
  if (batch->launched) cudaEventSynchronize(batch->last);
  r.camera = *cam;
  r.eye_sep = eye_sep;
  r.convergence = convergence;
  batch->reqs[i] = r;
  batch->args[i] = a;
  rt::BatchReq& q = batch->h_table[batch->pos[i]];
  const uint32_t tx = q.cam.tiles_x, ty = q.cam.tiles_y;
  q.cam = a.cam;
  q.cam.tiles_x = tx;
  q.cam.tiles_y = ty;
  return RT_OK;
}

int rt_batch_stats(rt_batch* batch, uint64_t* ray_counts, float* request_ms, rt_batch_config* cfg) {
  if (!batch) return fail(RT_ERR_INVALID_ARG, "batch is NULL");
  if (cfg) *cfg = batch->cfg;
  if (!batch->launched) {
    if (ray_counts) ray_counts[0] = ray_counts[1] = ray_counts[2] = 0;
    if (request_ms) for (uint32_t i = 0; i < batch->n; ++i) request_ms[i] = -1.f;
    return RT_OK;
  }
  cudaError_t e = cudaEventSynchronize(batch->last);
  if (e != cudaSuccess) return cuda_fail(e, "rt_batch_stats: wait");
  const int rc = check_status(batch);
  if (rc != RT_OK) return rc;
  if (ray_counts) {
    uint32_t c[rt::C_TOTAL];
    e = cudaMemcpy(c, batch->counters, sizeof c, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "rt_batch_stats: counters");
    ray_counts[0] = batch->primary_rays;
    ray_counts[1] = c[rt::C_SHADOW];
    ray_counts[2] = c[rt::C_REFL];
  }
  if (request_ms) {
    if (!batch->cfg.track_latency) {
      for (uint32_t i = 0; i < batch->n; ++i) request_ms[i] = -1.f;
    } else {
      std::vector<unsigned long long> t(batch->n + 1);
      e = cudaMemcpy(t.data(), batch->done_ns, t.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "rt_batch_stats: timestamps");
      const unsigned long long t0 = t[batch->n];
      for (uint32_t i = 0; i < batch->n; ++i) {
        const unsigned long long d = t[batch->pos[i]];
        request_ms[i] = d > t0 ? (float)((double)(d - t0) * 1e-6) : 0.f;
      }
    }
  }
  return RT_OK;
}

int rt_batch_autotune(rt_batch* batch, uint32_t reps, void* cuda_stream, rt_batch_config* chosen,
                      float* best_ms) {
  if (!batch || reps < 1 || reps > 1000) return fail(RT_ERR_INVALID_ARG, "batch is NULL or reps outside 1..1000");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "rt_batch_autotune: events");
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(cudaGetLastError(), "rt_batch_autotune: events"); }
  auto time_config = [&](const rt_batch_config& c, float& ms) -> int {
    int rc = apply_config(batch, c);
    if (rc != RT_OK) return rc;
    rc = rt_batch_launch(batch, st);                    // warm-up
    if (rc != RT_OK) return rc;
    std::vector<float> ts;
    for (uint32_t k = 0; k < reps; ++k) {
      cudaEventRecord(e0, st);
      rc = rt_batch_launch(batch, st);
      if (rc != RT_OK) return rc;
      cudaEventRecord(e1, st);
      const cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) return cuda_fail(e, "rt_batch_autotune: wait");
      float x = 0.f;
      cudaEventElapsedTime(&x, e0, e1);
      ts.push_back(x);
    }
    rc = check_status(batch);
    if (rc != RT_OK) return rc;
    std::sort(ts.begin(), ts.end());
    ms = ts[ts.size() / 2];
    return RT_OK;
  };
  rt_batch_config best = batch->cfg;
  float best_t = 0.f;
  int rc = time_config(best, best_t);
  const int occ = rt::batch_occupancy();
  const uint32_t tiles[6][2] = {{4, 4}, {8, 2}, {2, 8}, {8, 4}, {4, 8}, {16, 2}};
  for (int dim = 0; dim < 4 && rc == RT_OK; ++dim) {
    std::vector<rt_batch_config> cands;
    if (dim == 0) {
      for (auto& t : tiles) { rt_batch_config c = best; c.tile_w = t[0]; c.tile_h = t[1]; cands.push_back(c); }
    } else if (dim == 1) {
      for (int k : {occ, occ - 2, occ - 4})
        if (k >= 1) { rt_batch_config c = best; c.blocks_per_sm = (uint32_t)k; cands.push_back(c); }
    } else if (dim == 2) {
      for (uint32_t cap : {64u, 128u, 256u}) { rt_batch_config c = best; c.cap_r = cap; cands.push_back(c); }
    } else {
      for (uint32_t o : {0u, 1u, 2u}) { rt_batch_config c = best; c.order = o; cands.push_back(c); }
    }
    for (const rt_batch_config& c : cands) {
      if (!std::memcmp(&c, &best, sizeof c)) continue;
      float t = 0.f;
      rc = time_config(c, t);
      if (rc != RT_OK) break;
      if (t < best_t) { best = c; best_t = t; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != RT_OK) return rc;
  rc = apply_config(batch, best);
  if (rc != RT_OK) return rc;
  if (chosen) *chosen = batch->cfg;
  if (best_ms) *best_ms = best_t;
  return RT_OK;
}

}  // extern "C"
