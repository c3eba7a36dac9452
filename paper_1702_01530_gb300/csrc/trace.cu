// Stereo-pair ray tracing on the GPU (sm_103a): the hot path.
//
// Paper Sec. 3: the left and right channel are independent ("parallel level
// 1") and the pixels of a channel are traced in parallel ("parallel level 2");
// the image is split into parts processed by parallel workers (Figure 1).
// Here both eyes share one launch: persistent warps pull 32-ray batches from
// a global counter, and the primary batches are 8x4-pixel tiles that
// alternate left / right eye, so the two eyes' nearly identical rays touch
// the same BVH nodes close together in time.
//
// Per stereo pair (D = max_depth):
//   k_trace<PRIMARY>    primary rays of both eyes: generate, closest hit,
//                       shade; push shadow rays (queue S) and mirror rays
//                       (queue Q1)
//   k_shadow            any-hit over S; unblocked contributions accumulate
//   for d = 1..D: k_trace<REFLECT> over Q_d (push S, Q_{d+1}), k_shadow
//   k_resolve           fixed-point sums -> float RGB, clamp to [0,1]
//
// Colour sums are fixed-point uint32 per channel (atomic adds of
// round(value * 2^k)): integer addition is associative, so the image does
// not depend on the order in which shadow rays finish, and both eyes of a
// zero-separation pair are bitwise identical.
//
// Traversal (Table 1 of the paper: BVH trees): BVH2 nodes of 64 B with both
// child boxes, read as four 16-byte vector loads through the read-only path;
// slab tests in FP32 with fused multiply-adds and three-input min/max; the
// far child is pushed on a per-thread stack (depth <= 64 by construction of
// the radix tree over unique 64-bit keys), the near child is visited first.
// Each loop has an iteration bound; hitting it sets the error word.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_internal.cuh"

namespace rt {
namespace {

constexpr int kThreads = 128;
constexpr float kRobust = 1.00000036f;   // 1 + 2*gamma_3 (Ize 2013): conservative slab exit

__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

struct V3 { float x, y, z; };
__device__ __forceinline__ V3 v3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(V3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return {fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x)};
}
__device__ __forceinline__ V3 normalize(V3 a) { return a * rsqrtf(dot(a, a)); }
__device__ __forceinline__ V3 xyz(float4 f) { return {f.x, f.y, f.z}; }

__device__ __forceinline__ float safe_rcp(float x) {
  const float tiny = 8.271806e-25f;  // 2^-80
  return __frcp_rn(fabsf(x) > tiny ? x : copysignf(tiny, x));
}

struct WorkCount { uint32_t inner, sphere, tri; };

// Ray-sphere (d unit length). Stable form: disc = r^2 - |oc - b d|^2 keeps
// precision when the ray passes far from the centre relative to r; the two
// roots are q and c/q with q = -b - sign(b) sqrt(disc).
__device__ __forceinline__ bool hit_sphere(float4 p0, float r, V3 o, V3 d, float& t) {
  V3 oc = o - xyz(p0);
  float b = dot(oc, d);
  V3 f = oc - d * b;
  float r2 = r * r;
  float disc = r2 - dot(f, f);
  float cc = dot(oc, oc) - r2;
  float sq = sqrtf(fmaxf(disc, 0.f));
  float q = -b - copysignf(sq, b);
  float t0 = __fdividef(cc, q), t1 = q;
  float tn = fminf(t0, t1), tf = fmaxf(t0, t1);
  t = tn > 0.f ? tn : tf;
  return disc >= 0.f && t > 0.f;
}

// Moller-Trumbore, two-sided, edges inclusive (branch-free acceptance). The
// barycentric bounds are widened by kEdge so that a ray through the shared
// edge of two triangles cannot slip between them when FP32 rounding puts it
// just outside both (the band lies far inside the oracle's near-tie margin).
constexpr float kEdge = 1e-6f;
__device__ __forceinline__ bool hit_tri(float4 p0, float4 p1, float4 p2, V3 o, V3 d, float& t) {
  V3 e1 = xyz(p1), e2 = xyz(p2);
  V3 pv = cross(d, e2);
  float det = dot(e1, pv);
  float inv = __frcp_rn(det);
  V3 tv = o - xyz(p0);
  float u = dot(tv, pv) * inv;
  V3 qv = cross(tv, e1);
  float v = dot(d, qv) * inv;
  t = dot(e2, qv) * inv;
  return det != 0.f && u >= -kEdge && v >= -kEdge && u + v <= 1.f + kEdge && t > 0.f;
}

// BVH traversal. ANY = any-hit with t < tmax (returns true if blocked);
// otherwise closest hit with t <= t_best (equal t -> lower id), returns
// whether anything was hit.
template <bool ANY, bool COUNT>
__device__ __forceinline__ bool traverse(const DeviceScene& sc, V3 o, V3 d, float tmax,
                                         float& t_best, uint32_t& id_best, uint32_t& k_best,
                                         WorkCount& wc, uint32_t* err) {
  const V3 idir = v3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
  const V3 ood = v3(o.x * idir.x, o.y * idir.y, o.z * idir.z);
  int32_t stack[kStackSize];
  int sp = 0;
  const uint32_t n = sc.n_prims;
  int32_t node = n == 1 ? ~0 : 0;
  const uint32_t it_max = 2u * n + 64u;
  float tcur = ANY ? tmax : t_best;
  bool any = false;
  for (uint32_t it = 0;; ++it) {
    if (it >= it_max) { atomicOr(err, ERR_ITER); break; }
    if (node >= 0) {
      if ((uint32_t)node >= n - 1) { atomicOr(err, ERR_INDEX); break; }
      const float4* np = sc.nodes + 4 * (size_t)node;
      const float4 a = __ldg(np), b = __ldg(np + 1), c = __ldg(np + 2), e = __ldg(np + 3);
      if (COUNT) wc.inner++;
      const float l0x = fmaf(a.x, idir.x, -ood.x), h0x = fmaf(a.y, idir.x, -ood.x);
      const float l0y = fmaf(a.z, idir.y, -ood.y), h0y = fmaf(a.w, idir.y, -ood.y);
      const float l0z = fmaf(c.x, idir.z, -ood.z), h0z = fmaf(c.y, idir.z, -ood.z);
      const float l1x = fmaf(b.x, idir.x, -ood.x), h1x = fmaf(b.y, idir.x, -ood.x);
      const float l1y = fmaf(b.z, idir.y, -ood.y), h1y = fmaf(b.w, idir.y, -ood.y);
      const float l1z = fmaf(c.z, idir.z, -ood.z), h1z = fmaf(c.w, idir.z, -ood.z);
      const float in0 = fmax3(fminf(l0x, h0x), fminf(l0y, h0y), fmaxf(fminf(l0z, h0z), 0.f));
      const float out0 = fmin3(fmaxf(l0x, h0x), fmaxf(l0y, h0y), fminf(fmaxf(l0z, h0z), tcur));
      const float in1 = fmax3(fminf(l1x, h1x), fminf(l1y, h1y), fmaxf(fminf(l1z, h1z), 0.f));
      const float out1 = fmin3(fmaxf(l1x, h1x), fmaxf(l1y, h1y), fminf(fmaxf(l1z, h1z), tcur));
      const bool hit0 = in0 <= out0 * kRobust;
      const bool hit1 = in1 <= out1 * kRobust;
      const int32_t cl = __float_as_int(e.x), cr = __float_as_int(e.y);
      if (hit0 && hit1) {
        const bool swap = in1 < in0;
        if (sp >= kStackSize) { atomicOr(err, ERR_STACK); break; }
        stack[sp++] = swap ? cl : cr;
        node = swap ? cr : cl;
        continue;
      }
      if (hit0 | hit1) { node = hit0 ? cl : cr; continue; }
    } else {
      const uint32_t k = (uint32_t)~node;
      if (k >= n) { atomicOr(err, ERR_INDEX); break; }
      const float4* pp = sc.prims + 3 * (size_t)k;
      const float4 p0 = __ldg(pp), p1 = __ldg(pp + 1);
      const uint32_t id = __float_as_uint(p0.w);
      float t;
      bool h;
      if (id < sc.n_spheres) {
        if (COUNT) wc.sphere++;
        h = hit_sphere(p0, p1.x, o, d, t);
      } else {
        if (COUNT) wc.tri++;
        h = hit_tri(p0, p1, __ldg(pp + 2), o, d, t);
      }
      if (ANY) {
        if (h && t < tmax) { any = true; break; }
      } else if (h && (t < tcur || (t == tcur && id < id_best))) {
        tcur = t;
        id_best = id;
        k_best = k;
        any = true;
      }
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  if (!ANY) t_best = tcur;
  return any;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// warp-aggregated reservation of one slot per thread with pred set
__device__ __forceinline__ uint32_t reserve(uint32_t* ctr, bool pred, uint32_t& slot) {
  const uint32_t mask = __ballot_sync(__activemask(), pred);
  if (!pred) return 0;
  const uint32_t leader = __ffs(mask) - 1;
  uint32_t base = 0;
  if (lane_id() == leader) base = atomicAdd(ctr, (uint32_t)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  slot = base + __popc(mask & ((1u << lane_id()) - 1u));
  return 1;
}

__device__ __forceinline__ void accumulate(uint32_t* acc, uint32_t pix, float r, float g, float b,
                                           float scale) {
  uint32_t* p = acc + 3 * (size_t)pix;
  atomicAdd(p + 0, __float2uint_rn(r * scale));
  atomicAdd(p + 1, __float2uint_rn(g * scale));
  atomicAdd(p + 2, __float2uint_rn(b * scale));
}

struct KParams {
  RenderArgs a;
  uint32_t* accum;
  const float4* qin;
  float4* qout;
  float4* shadow;
  uint32_t* counters;
  uint64_t cap_rays, cap_shadow;
  uint32_t depth;
};

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

// Closest-hit + shading kernel. PRIMARY: rays come from the camera, one
// 8x4-pixel tile per 32 slots, tiles alternating eyes. Otherwise the rays
// are read from the reflection queue of this depth.
template <bool PRIMARY, bool COUNT>
__global__ void __launch_bounds__(kThreads) k_trace(KParams kp) {
  const RenderArgs& a = kp.a;
  const CameraParams& cam = a.cam;
  const uint32_t P = cam.W * cam.H;
  // queue lengths are clamped to the capacity: entries past it were never written
  const uint32_t n = PRIMARY ? 2u * cam.tiles_x * cam.tiles_y * 32u
                             : (uint32_t)min((uint64_t)*(volatile uint32_t*)&kp.counters[C_QLEN + kp.depth],
                                             kp.cap_rays);
  uint32_t* work_ctr = &kp.counters[C_WORK + 2 * kp.depth];
  WorkCount wc = {0, 0, 0};
  for (;;) {
    uint32_t base = 0;
    if (lane_id() == 0) base = atomicAdd(work_ctr, 32u);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base >= n) break;
    const uint32_t idx = base + lane_id();
    bool active = idx < n;
    V3 o, d, w = v3(1.f, 1.f, 1.f);
    uint32_t pix = 0;
    if (PRIMARY) {
      const uint32_t tile = idx >> 5, ln = idx & 31u;
      const uint32_t eye = tile & 1u, tt = tile >> 1;
      const uint32_t px = (tt % cam.tiles_x) * 8u + (ln & 7u);
      const uint32_t py = (tt / cam.tiles_x) * 4u + (ln >> 3);
      active = active && px < cam.W && py < cam.H;
      pix = eye * P + py * cam.W + px;
      const float nx = (2.f * ((float)px + 0.5f) / (float)cam.W - 1.f) * cam.tan_x;
      const float ny = (1.f - 2.f * ((float)py + 0.5f) / (float)cam.H) * cam.tan_y;
      const V3 E = v3(cam.eye[0], cam.eye[1], cam.eye[2]);
      const V3 R = v3(cam.right[0], cam.right[1], cam.right[2]);
      const V3 U = v3(cam.up[0], cam.up[1], cam.up[2]);
      const V3 F = v3(cam.fwd[0], cam.fwd[1], cam.fwd[2]);
      const V3 Q = E + (F + R * nx + U * ny) * cam.zc;
      o = E + R * (eye ? cam.half_sep : -cam.half_sep);
      d = normalize(Q - o);
    } else if (active) {
      const float4 q0 = kp.qin[3 * (size_t)idx], q1 = kp.qin[3 * (size_t)idx + 1],
                   q2 = kp.qin[3 * (size_t)idx + 2];
      o = xyz(q0);
      pix = __float_as_uint(q0.w);
      d = xyz(q1);
      w = xyz(q2);
    }
    float t = INFINITY;
    uint32_t id = RT_MISS_ID, k = 0;
    bool hit = false;
    if (active) hit = traverse<false, COUNT>(a.sc, o, d, INFINITY, t, id, k, wc, a.err);

    // ------------------------------------------------------------ shading
    float amb_r = 0.f, amb_g = 0.f, amb_b = 0.f;
    V3 p = v3(0.f, 0.f, 0.f), nrm = v3(0.f, 0.f, 1.f), o2;
    float4 mat = make_float4(0.f, 0.f, 0.f, 0.f);
    float eps = 0.f;
    if (active) {
      if (!hit) {
        amb_r = w.x * kBgR; amb_g = w.y * kBgG; amb_b = w.z * kBgB;
      } else {
        const float4* pp = a.sc.prims + 3 * (size_t)k;
        const float4 p0 = __ldg(pp), p1 = __ldg(pp + 1);
        p = o + d * t;
        uint32_t mid = __float_as_uint(p1.w);
        if (id < a.sc.n_spheres) {
          nrm = (p - xyz(p0)) * (1.f / p1.x);
        } else {
          nrm = normalize(cross(xyz(p1), xyz(__ldg(pp + 2))));
        }
        if (dot(nrm, d) > 0.f) nrm = nrm * -1.f;
        if (mid >= a.sc.n_mats) { atomicOr(a.err, ERR_INDEX); mid = 0; }
        mat = __ldg(a.sc.mats + mid);
        const float kd = (1.f - mat.w) * kAmbient;
        amb_r = w.x * kd * mat.x; amb_g = w.y * kd * mat.y; amb_b = w.z * kd * mat.z;
        eps = 1e-4f * fmaxf(1.f, fmax3(fabsf(p.x), fabsf(p.y), fabsf(p.z)));
      }
      accumulate(kp.accum, pix, amb_r, amb_g, amb_b, a.color_scale);
    }
    o2 = p + nrm * eps;
    // shadow rays: one per light facing the surface
    const uint32_t L = a.sc.n_lights;
    for (uint32_t l = 0; l < L; ++l) {
      bool emit = false;
      V3 lh = v3(0.f, 0.f, 1.f);
      float ld = 0.f, ndl = 0.f;
      if (active && hit) {
        const float4 lp = __ldg(a.sc.lights + l);
        const V3 lv = xyz(lp) - o2;
        const float inv = rsqrtf(dot(lv, lv));
        ld = dot(lv, lv) * inv;
        lh = lv * inv;
        ndl = dot(nrm, lh);
        emit = ndl > 0.f;
        ndl *= lp.w * (1.f - mat.w);
      }
      uint32_t slot;
      if (reserve(&kp.counters[C_SLEN + kp.depth], emit, slot)) {
        if (slot < kp.cap_shadow) {
          float4* s = kp.shadow + 3 * (size_t)slot;
          s[0] = make_float4(o2.x, o2.y, o2.z, __uint_as_float(pix));
          s[1] = make_float4(lh.x, lh.y, lh.z, ld - eps);
          s[2] = make_float4(w.x * ndl * mat.x, w.y * ndl * mat.y, w.z * ndl * mat.z, 0.f);
        } else {
          atomicOr(a.err, ERR_QUEUE);
        }
      }
    }
    // mirror ray
    const bool refl = active && hit && mat.w > 0.f && kp.depth < a.max_depth;
    uint32_t slot;
    if (reserve(&kp.counters[C_QLEN + kp.depth + 1], refl, slot)) {
      if (slot < kp.cap_rays) {
        V3 rd = normalize(d - nrm * (2.f * dot(d, nrm)));
        float4* q = kp.qout + 3 * (size_t)slot;
        q[0] = make_float4(o2.x, o2.y, o2.z, __uint_as_float(pix));
        q[1] = make_float4(rd.x, rd.y, rd.z, 0.f);
        q[2] = make_float4(w.x * mat.w, w.y * mat.w, w.z * mat.w, 0.f);
      } else {
        atomicOr(a.err, ERR_QUEUE);
      }
    }
    if (PRIMARY && active) {
      const uint32_t eye = pix >= P;
      const uint32_t pi = pix - eye * P;
      uint32_t* hid = eye ? a.hit_R : a.hit_L;
      float* dep = eye ? a.depth_R : a.depth_L;
      if (hid) hid[pi] = id;
      if (dep) dep[pi] = hit ? t * dot(d, v3(cam.fwd[0], cam.fwd[1], cam.fwd[2])) : INFINITY;
    }
  }
  if (COUNT) flush_work(wc, a.work, PRIMARY ? 0 : 2);
}

// Any-hit over the shadow queue of this depth; unblocked rays add their
// precomputed contribution to the pixel.
template <bool COUNT>
__global__ void __launch_bounds__(kThreads) k_shadow(KParams kp) {
  const RenderArgs& a = kp.a;
  const uint32_t n = (uint32_t)min((uint64_t)*(volatile uint32_t*)&kp.counters[C_SLEN + kp.depth],
                                   kp.cap_shadow);
  uint32_t* work_ctr = &kp.counters[C_WORK + 2 * kp.depth + 1];
  WorkCount wc = {0, 0, 0};
  for (;;) {
    uint32_t base = 0;
    if (lane_id() == 0) base = atomicAdd(work_ctr, 32u);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base >= n) break;
    const uint32_t idx = base + lane_id();
    if (idx >= n) continue;
    const float4* s = kp.shadow + 3 * (size_t)idx;
    const float4 s0 = s[0], s1 = s[1];
    float tb = 0.f;
    uint32_t id = 0, k = 0;
    const bool blocked = traverse<true, COUNT>(a.sc, xyz(s0), xyz(s1), s1.w, tb, id, k, wc, a.err);
    if (!blocked) {
      const float4 s2 = s[2];
      accumulate(kp.accum, __float_as_uint(s0.w), s2.x, s2.y, s2.z, a.color_scale);
    }
  }
  if (COUNT) flush_work(wc, a.work, 1);
}

__global__ void k_resolve(const uint32_t* __restrict__ acc, float* __restrict__ out_L,
                          float* __restrict__ out_R, uint32_t n3, float inv_scale) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * n3; i += gridDim.x * blockDim.x) {
    const float v = fminf(1.f, (float)acc[i] * inv_scale);
    if (i < n3) out_L[i] = v; else out_R[i - n3] = v;
  }
}

__global__ void k_counts(const uint32_t* counters, uint32_t max_depth, uint64_t primary,
                         uint64_t* out) {
  if (threadIdx.x != 0) return;
  uint64_t sh = 0, rf = 0;
  for (uint32_t d = 0; d <= max_depth; ++d) sh += counters[C_SLEN + d];
  for (uint32_t d = 1; d <= max_depth; ++d) rf += counters[C_QLEN + d];
  out[0] = primary;
  out[1] = sh;
  out[2] = rf;
}

template <typename K>
int grid_for(K kernel) {
  static int cached = 0;
  if (!cached) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0);
    cached = num_sms() * (per_sm > 0 ? per_sm : 1);
  }
  return cached;
}

template <bool COUNT>
cudaError_t render_impl(const RenderArgs& a, Workspace& ws, cudaStream_t st) {
  const uint64_t P = (uint64_t)a.cam.W * a.cam.H;
  KParams kp;
  kp.a = a;
  kp.accum = ws.accum;
  kp.shadow = ws.shadow;
  kp.counters = ws.counters;
  kp.cap_rays = ws.cap_rays;
  kp.cap_shadow = ws.cap_shadow;
  ws.n_ev = 0;
  auto mark = [&](int stage) {  // stage timing: an event after each stage
    if (!ws.profile) return;
    ws.ev_stage[ws.n_ev] = stage;
    cudaEventRecord(ws.ev[ws.n_ev++], st);
  };
  mark(-1);
  cudaMemsetAsync(ws.counters, 0, C_TOTAL * sizeof(uint32_t), st);
  cudaMemsetAsync(ws.accum, 0, 2 * P * 3 * sizeof(uint32_t), st);
  if (a.work) cudaMemsetAsync(a.work, 0, 9 * sizeof(uint64_t), st);
  mark(ST_CLEAR);
  for (uint32_t d = 0; d <= a.max_depth; ++d) {
    kp.depth = d;
    kp.qin = ws.queue[d & 1];
    kp.qout = ws.queue[(d + 1) & 1];
    if (d == 0) {
      k_trace<true, COUNT><<<grid_for(k_trace<true, COUNT>), kThreads, 0, st>>>(kp);
      mark(ST_PRIMARY);
    } else {
      k_trace<false, COUNT><<<grid_for(k_trace<false, COUNT>), kThreads, 0, st>>>(kp);
      mark(ST_REFLECT);
    }
    k_shadow<COUNT><<<grid_for(k_shadow<COUNT>), kThreads, 0, st>>>(kp);
    mark(d == 0 ? ST_SHADOW0 : ST_SHADOWN);
  }
  const uint32_t n3 = (uint32_t)(P * 3);
  k_resolve<<<num_sms() * 8, 256, 0, st>>>(ws.accum, a.out_L, a.out_R, n3, 1.f / a.color_scale);
  mark(ST_RESOLVE);
  if (a.ray_counts) k_counts<<<1, 32, 0, st>>>(ws.counters, a.max_depth, 2 * P, a.ray_counts);
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

cudaError_t render(const RenderArgs& a, Workspace& ws, cudaStream_t st) {
  return a.work ? render_impl<true>(a, ws, st) : render_impl<false>(a, ws, st);
}

}  // namespace rt
