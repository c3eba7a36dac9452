// Stereo-pair ray tracing on the GPU (sm_103a): the hot path.
//
// Paper Sec. 3: the left and right channel are independent ("parallel level
// 1") and the pixels of a channel are traced in parallel ("parallel level 2");
// the image is split into parts processed by parallel workers (Figure 1).
// Here both eyes share one persistent launch: warps pull 8x4-pixel tiles from
// a global counter, tiles alternating left / right eye, so the two eyes'
// nearly identical rays touch the same BVH nodes close together in time.
//
// Per stereo pair:
//   k_render   one persistent kernel. Every warp owns two small wavefront
//              queues in global memory (L2-resident): shadow rays and mirror
//              rays produced by its own shading. Each round the warp picks,
//              warp-uniformly, 32 queued shadow rays (any-hit), else 32
//              queued mirror rays (closest hit + shade), else a new primary
//              tile (generate + closest hit + shade); when the tiles are gone
//              it drains its queues. Rounds are full warps except the final
//              drain, no ray waits for a later launch, and there is one
//              launch tail per frame instead of one per bounce depth.
//   k_resolve  fixed-point sums -> float RGB, clamp to [0,1]
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

// Tuning knobs (compile-time): RT_MIN_BLOCKS = minimum resident blocks per
// SM requested from the register allocator (0 = no request; 10 measured
// best on GB300: 48 registers, 40 warps per SM); RT_WHILE_WHILE = 1
// postpones the first leaf a ray meets and keeps descending until every
// active lane of the warp holds a leaf, so the leaf tests of a warp run
// together instead of interleaving with node visits (the "while-while" loop
// of Aila & Laine, HPG 2009) -- 20 % slower here with one primitive per leaf,
// hence off by default.
#ifndef RT_MIN_BLOCKS
#define RT_MIN_BLOCKS 10
#endif
#ifndef RT_WHILE_WHILE
#define RT_WHILE_WHILE 0
#endif
constexpr int kStack4 = 100;   // 3 pushes per 4-wide level, <= 33 levels
// shared-memory treelet: 4-wide levels staged per block (RT_TREELET_DEPTH
// levels, at most 1 + 4 + 16 + 64 = 85 nodes for depth 4)
#ifndef RT_TREELET_DEPTH
#define RT_TREELET_DEPTH 2
#endif
constexpr int kMaxTopBytes = 85 * 7 * 16;
// shadow rounds take the warp's whole shadow queue and every lane fetches its
// next entry as soon as its ray finishes (per-warp counter in shared memory);
// measured 1.55 vs 1.53 ms per 1080p blob pair: off by default
#ifndef RT_SHADOW_REFILL
#define RT_SHADOW_REFILL 0
#endif
// binary traversal keeps the top of its stack in a register: a pop hands
// the register over at once and reloads it from local memory in the
// background, so the pop and the next node fetch do not wait in series;
// measured 1.60 vs 1.53 ms per 1080p blob pair: off by default
#ifndef RT_STACK_TOP_REG
#define RT_STACK_TOP_REG 0
#endif
// 4-wide closest-hit traversal pushes the other hit children farthest first
#ifndef RT_ORDERED_PUSH
#define RT_ORDERED_PUSH 0
#endif
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
  constexpr int32_t kNone = 0x7FFFFFFF;        // no node: empty stack
  const V3 idir = v3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
  const V3 ood = v3(o.x * idir.x, o.y * idir.y, o.z * idir.z);
  int32_t stack[kStackSize];
  int sp = 0;
  int32_t stop = kNone;                         // top of the stack (register copy)
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
        const int32_t far = swap ? cl : cr;
        if (RT_STACK_TOP_REG) {
          if (stop != kNone) {
            if (sp >= kStackSize) { atomicOr(err, ERR_STACK); break; }
            stack[sp++] = stop;
          }
          stop = far;
        } else {
          if (sp >= kStackSize) { atomicOr(err, ERR_STACK); break; }
          stack[sp++] = far;
        }
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
    if (RT_STACK_TOP_REG) {
      if (stop == kNone) break;
      node = stop;
      stop = sp ? stack[--sp] : kNone;
    } else {
      if (sp == 0) break;
      node = stack[--sp];
    }
  }
  if (!ANY) t_best = tcur;
  return any;
}

// 4-wide traversal: one fetch of 7 float4 tests four child boxes; the
// nearest hit child is visited next and the other hit children are pushed.
// The first sc.n_top nodes are read from the shared-memory copy `top`.
template <bool ANY>
__device__ __forceinline__ bool traverse4(const DeviceScene& sc, const float4* top, V3 o, V3 d,
                                          float tmax, float& t_best, uint32_t& id_best,
                                          uint32_t& k_best, uint32_t* err) {
  const V3 idir = v3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
  const V3 ood = v3(o.x * idir.x, o.y * idir.y, o.z * idir.z);
  int32_t stack[kStack4];
  int sp = 0;
  const uint32_t n = sc.n_prims;
  int32_t node = n == 1 ? ~0 : 0;
  const uint32_t it_max = 2u * n + 64u;
  float tcur = ANY ? tmax : t_best;
  bool any = false;
  for (uint32_t it = 0;; ++it) {
    if (it >= it_max) { atomicOr(err, ERR_ITER); break; }
    if (node >= 0) {
      if ((uint32_t)node >= sc.n4) { atomicOr(err, ERR_INDEX); break; }
      float4 lx, hx, ly, hy, lz, hz, cc;
      if ((uint32_t)node < sc.n_top) {             // shared-memory treelet
        const float4* np = top + 7 * node;
        lx = np[0]; hx = np[1]; ly = np[2]; hy = np[3]; lz = np[4]; hz = np[5]; cc = np[6];
      } else {                                     // read-only global path
        const float4* np = sc.nodes4 + 7 * (size_t)node;
        lx = __ldg(np); hx = __ldg(np + 1); ly = __ldg(np + 2); hy = __ldg(np + 3);
        lz = __ldg(np + 4); hz = __ldg(np + 5); cc = __ldg(np + 6);
      }
      float tin[4];
      bool hit[4];
#define RT_SLAB(c, LX, HX, LY, HY, LZ, HZ)                                                  \
      {                                                                                     \
        const float ax = fmaf(LX, idir.x, -ood.x), bx = fmaf(HX, idir.x, -ood.x);           \
        const float ay = fmaf(LY, idir.y, -ood.y), by = fmaf(HY, idir.y, -ood.y);           \
        const float az = fmaf(LZ, idir.z, -ood.z), bz = fmaf(HZ, idir.z, -ood.z);           \
        tin[c] = fmax3(fminf(ax, bx), fminf(ay, by), fmaxf(fminf(az, bz), 0.f));             \
        const float tout = fmin3(fmaxf(ax, bx), fmaxf(ay, by), fminf(fmaxf(az, bz), tcur));  \
        hit[c] = tin[c] <= tout * kRobust;                                                  \
      }
      RT_SLAB(0, lx.x, hx.x, ly.x, hy.x, lz.x, hz.x)
      RT_SLAB(1, lx.y, hx.y, ly.y, hy.y, lz.y, hz.y)
      RT_SLAB(2, lx.z, hx.z, ly.z, hy.z, lz.z, hz.z)
      RT_SLAB(3, lx.w, hx.w, ly.w, hy.w, lz.w, hz.w)
#undef RT_SLAB
      const int32_t ch[4] = {__float_as_int(cc.x), __float_as_int(cc.y), __float_as_int(cc.z),
                             __float_as_int(cc.w)};
#pragma unroll
      for (int c = 0; c < 4; ++c) hit[c] = hit[c] && ch[c] != kEmptyChild;  // unused slots
      int bi = -1;
      float best = INFINITY;
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (hit[c] && (ANY ? bi < 0 : tin[c] < best)) { best = tin[c]; bi = c; }
      if (bi >= 0) {
        // the other hit children, farthest pushed first (closest-hit rays)
        float t4[4];
        int32_t c4[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          t4[c] = (hit[c] && c != bi) ? tin[c] : -INFINITY;
          c4[c] = ch[c];
        }
        if (!ANY && RT_ORDERED_PUSH) {
#define RT_CAS(i, j)                                                              \
          if (t4[i] < t4[j]) {                                                    \
            const float tt = t4[i]; t4[i] = t4[j]; t4[j] = tt;                    \
            const int32_t cx = c4[i]; c4[i] = c4[j]; c4[j] = cx;                  \
          }
          RT_CAS(0, 1) RT_CAS(2, 3) RT_CAS(0, 2) RT_CAS(1, 3) RT_CAS(1, 2)
#undef RT_CAS
        }
        bool overflow = false;
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (t4[c] > -INFINITY) {
            if (sp < kStack4) stack[sp++] = c4[c];
            else overflow = true;
          }
        if (overflow) { atomicOr(err, ERR_STACK); break; }
        node = ch[bi];
        continue;
      }
    } else {
      const uint32_t k = (uint32_t)~node;
      if (k >= n) { atomicOr(err, ERR_INDEX); break; }
      const float4* pp = sc.prims + 3 * (size_t)k;
      const float4 p0 = __ldg(pp), p1 = __ldg(pp + 1);
      const uint32_t id = __float_as_uint(p0.w);
      float t;
      bool h;
      if (id < sc.n_spheres) h = hit_sphere(p0, p1.x, o, d, t);
      else h = hit_tri(p0, p1, __ldg(pp + 2), o, d, t);
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

#if RT_WHILE_WHILE
// Same traversal with postponed leaves. Internal nodes are visited until
// every active lane of the warp holds one pending leaf (or has finished);
// then the pending leaves (and any leaves that follow directly) are tested.
template <bool ANY, bool COUNT>
__device__ __forceinline__ bool traverse_ww(const DeviceScene& sc, V3 o, V3 d, float tmax,
                                            float& t_best, uint32_t& id_best, uint32_t& k_best,
                                            WorkCount& wc, uint32_t* err) {
  constexpr int32_t kDone = 0x7FFFFFFF;   // larger than any internal node index
  const V3 idir = v3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
  const V3 ood = v3(o.x * idir.x, o.y * idir.y, o.z * idir.z);
  int32_t stack[kStackSize];
  int sp = 0;
  const uint32_t n = sc.n_prims;
  int32_t node = n == 1 ? ~0 : 0;
  int32_t leaf = 0;
  const uint32_t it_max = 2u * n + 64u;
  uint32_t it = 0;
  float tcur = ANY ? tmax : t_best;
  bool any = false;
  if (node < 0) { leaf = node; node = kDone; }
  while (node != kDone || leaf != 0) {
    while ((uint32_t)node < (uint32_t)kDone) {   // node >= 0 and not done
      if (++it > it_max) { atomicOr(err, ERR_ITER); node = kDone; leaf = 0; break; }
      if ((uint32_t)node >= n - 1) { atomicOr(err, ERR_INDEX); node = kDone; leaf = 0; break; }
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
        if (sp >= kStackSize) { atomicOr(err, ERR_STACK); node = kDone; leaf = 0; break; }
        stack[sp++] = swap ? cl : cr;
        node = swap ? cr : cl;
      } else if (hit0 | hit1) {
        node = hit0 ? cl : cr;
      } else {
        node = sp ? stack[--sp] : kDone;
      }
      if (node < 0 && leaf == 0) {           // postpone this leaf, keep descending
        leaf = node;
        node = sp ? stack[--sp] : kDone;
      }
      if (!__any_sync(__activemask(), leaf == 0)) break;
    }
    while (leaf < 0) {
      if (++it > it_max) { atomicOr(err, ERR_ITER); node = kDone; leaf = 0; break; }
      const uint32_t k = (uint32_t)~leaf;
      if (k >= n) { atomicOr(err, ERR_INDEX); node = kDone; leaf = 0; break; }
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
        if (h && t < tmax) { any = true; node = kDone; leaf = 0; break; }
      } else if (h && (t < tcur || (t == tcur && id < id_best))) {
        tcur = t;
        id_best = id;
        k_best = k;
        any = true;
      }
      leaf = 0;
      if (node < 0) {                         // the next node is a leaf too
        leaf = node;
        node = sp ? stack[--sp] : kDone;
      }
    }
  }
  if (!ANY) t_best = tcur;
  return any;
}
#endif

// The instrumented (COUNT) and the requested binary traversal walk the
// binary radix tree, whose node visits define the algorithmic work; the
// production path walks the 4-wide tree (the same leaves, the same hits).
template <bool ANY, bool COUNT, bool WIDE>
__device__ __forceinline__ bool trace_ray(const DeviceScene& sc, const float4* top, V3 o, V3 d,
                                          float tmax, float& t_best, uint32_t& id_best,
                                          uint32_t& k_best, WorkCount& wc, uint32_t* err) {
  if (WIDE && !COUNT) return traverse4<ANY>(sc, top, o, d, tmax, t_best, id_best, k_best, err);
#if RT_WHILE_WHILE
  return traverse_ww<ANY, COUNT>(sc, o, d, tmax, t_best, id_best, k_best, wc, err);
#else
  return traverse<ANY, COUNT>(sc, o, d, tmax, t_best, id_best, k_best, wc, err);
#endif
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

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
  float4* wq;          // warp queues: per warp cap_s shadow then cap_r mirror entries
  uint32_t* counters;
  uint32_t cap_s, cap_r;
  uint32_t n_tiles;    // 2 * tiles_x * tiles_y
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

enum Mode : int { M_SHADOW = 0, M_PRIMARY = 1, M_MIRROR = 2 };

// Shadow queue entry: (origin | pixel) (direction | t_max) (contribution | 0)
// Mirror queue entry: (origin | pixel) (direction | depth) (weight | 0)
template <bool COUNT, bool WIDE>
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
  __shared__ uint32_t next_shadow[kThreads / 32];   // per-warp shadow-queue cursor
  if (WIDE && !COUNT) {
    for (uint32_t i = threadIdx.x; i < 7u * a.sc.n_top; i += blockDim.x) top[i] = a.sc.nodes4[i];
    __syncthreads();
  }
  const CameraParams& cam = a.cam;
  const uint32_t P = cam.W * cam.H;
  const uint32_t lane = lane_id();
  const uint32_t lt_mask = (1u << lane) - 1u;
  const size_t gwarp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  float4* const S = kp.wq + gwarp * 3 * (size_t)(kp.cap_s + kp.cap_r);
  float4* const R = S + 3 * (size_t)kp.cap_s;
  uint32_t nS = 0, nR = 0;          // warp-uniform queue fills
  uint32_t made_s = 0, made_r = 0;  // rays this warp enqueued
  bool tiles_left = true;
  const uint32_t plist_n = a.plist_n_dev ? *a.plist_n_dev : a.plist_n;
  const uint32_t n_tiles = a.plist ? (plist_n + 31u) / 32u : kp.n_tiles;
  WorkCount wc_p = {0, 0, 0}, wc_s = {0, 0, 0}, wc_r = {0, 0, 0};
  const uint32_t L = a.sc.n_lights;

  for (uint32_t round = 0;; ++round) {
    if (round > (1u << 30)) { if (lane == 0) atomicOr(a.err, ERR_ITER); break; }
    // ---------------------------------------------- warp-uniform schedule
    int mode;
    uint32_t take = 0, base = 0, tile = 0;
    if (nS >= 32) {
      mode = M_SHADOW;
      if (RT_SHADOW_REFILL) { take = nS; base = 0; nS = 0; }
      else { take = 32; nS -= 32; base = nS; }
    }
    else if (nR >= 32) { mode = M_MIRROR; take = 32; nR -= 32; base = nR; }
    else if (tiles_left) {
      uint32_t t = 0;
      if (lane == 0) t = atomicAdd(&kp.counters[C_TILE], 1u);
      t = __shfl_sync(0xFFFFFFFFu, t, 0);
      if (t >= n_tiles) { tiles_left = false; continue; }
      mode = M_PRIMARY; tile = t;
    }
    else if (nS > 0) { mode = M_SHADOW; take = nS; base = 0; nS = 0; }
    else if (nR > 0) { mode = M_MIRROR; take = nR; base = 0; nR = 0; }
    else break;

    if (mode == M_SHADOW) {
      // ------------------------------------------------ any-hit round
      if (RT_SHADOW_REFILL && lane == 0) next_shadow[threadIdx.x >> 5] = 32u;
      __syncwarp();
      uint32_t i = lane;
      while (i < take) {
        const float4* e = S + 3 * (size_t)(base + i);
        const float4 s0 = e[0], s1 = e[1];
        float tb = 0.f;
        uint32_t id = 0, k = 0;
        const bool blocked = trace_ray<true, COUNT, WIDE>(a.sc, top, xyz(s0), xyz(s1), s1.w, tb, id, k, wc_s, a.err);
        if (!blocked) {
          const float4 s2 = e[2];
          accumulate(kp.accum, __float_as_uint(s0.w), s2.x, s2.y, s2.z, a.color_scale);
        }
        i = RT_SHADOW_REFILL ? atomicAdd(&next_shadow[threadIdx.x >> 5], 1u) : take;
      }
      __syncwarp();
      continue;
    }

    // ------------------------------------------- closest hit + shading
    bool active;
    V3 o, d, w = v3(1.f, 1.f, 1.f);
    uint32_t pix = 0, depth = 0;
    if (mode == M_PRIMARY) {
      uint32_t eye, px, py;
      if (a.plist) {                       // an explicit pixel list (masked retrace)
        const uint32_t i = tile * 32u + lane;
        active = i < plist_n;
        pix = active ? a.plist[i] : 0u;
        if (pix >= 2 * P) { active = false; pix = 0u; }
        eye = pix >= P;
        const uint32_t pi = pix - eye * P;
        py = pi / cam.W;
        px = pi - py * cam.W;
      } else {                             // 8x4 tiles, alternating eyes when both are traced
        const uint32_t tt = a.eyes == 3u ? tile >> 1 : tile;
        eye = a.eyes == 3u ? (tile & 1u) : (a.eyes == 2u ? 1u : 0u);
        px = (tt % cam.tiles_x) * 8u + (lane & 7u);
        py = (tt / cam.tiles_x) * 4u + (lane >> 3);
        active = px < cam.W && py < cam.H;
        pix = eye * P + py * cam.W + px;
      }
      const float nx = (2.f * ((float)px + 0.5f) / (float)cam.W - 1.f) * cam.tan_x;
      const float ny = (1.f - 2.f * ((float)py + 0.5f) / (float)cam.H) * cam.tan_y;
      const V3 E = v3(cam.eye[0], cam.eye[1], cam.eye[2]);
      const V3 Rt = v3(cam.right[0], cam.right[1], cam.right[2]);
      const V3 U = v3(cam.up[0], cam.up[1], cam.up[2]);
      const V3 F = v3(cam.fwd[0], cam.fwd[1], cam.fwd[2]);
      const V3 Q = E + (F + Rt * nx + U * ny) * cam.zc;
      o = E + Rt * (eye ? cam.half_sep : -cam.half_sep);
      d = normalize(Q - o);
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
      }
      __syncwarp();  // every lane has read its entry before the slots are refilled
    }
    float t = INFINITY;
    uint32_t id = RT_MISS_ID, k = 0;
    bool hit = false;
    if (active)
      hit = trace_ray<false, COUNT, WIDE>(a.sc, top, o, d, INFINITY, t, id, k,
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
        const float4* pp = a.sc.prims + 3 * (size_t)k;
        const float4 p0 = __ldg(pp), p1 = __ldg(pp + 1);
        p = o + d * t;
        uint32_t mid = __float_as_uint(p1.w);
        if (id < a.sc.n_spheres) nrm = (p - xyz(p0)) * (1.f / p1.x);
        else nrm = normalize(cross(xyz(p1), xyz(__ldg(pp + 2))));
        if (dot(nrm, d) > 0.f) nrm = nrm * -1.f;
        if (mid >= a.sc.n_mats) { atomicOr(a.err, ERR_INDEX); mid = 0; }
        mat = __ldg(a.sc.mats + mid);
        const float kd = (1.f - mat.w) * kAmbient;
        ar = w.x * kd * mat.x; ag = w.y * kd * mat.y; ab = w.z * kd * mat.z;
        eps = 1e-4f * fmaxf(1.f, fmax3(fabsf(p.x), fabsf(p.y), fabsf(p.z)));
      }
      accumulate(kp.accum, pix, ar, ag, ab, a.color_scale);
    }
    const bool lit = active && hit;
    const V3 o2 = p + nrm * eps;
    // shadow rays into this warp's queue, one per light facing the surface
    for (uint32_t l = 0; l < L; ++l) {
      bool emit = false;
      V3 lh = v3(0.f, 0.f, 1.f);
      float ld = 0.f, ndl = 0.f;
      if (lit) {
        const float4 lp = __ldg(a.sc.lights + l);
        const V3 lv = xyz(lp) - o2;
        const float inv = rsqrtf(dot(lv, lv));
        ld = dot(lv, lv) * inv;
        lh = lv * inv;
        ndl = dot(nrm, lh);
        emit = ndl > 0.f;
        ndl *= lp.w * (1.f - mat.w);
      }
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
      const V3 rd = normalize(d - nrm * (2.f * dot(d, nrm)));
      float4* e = R + 3 * (size_t)rslot;
      e[0] = make_float4(o2.x, o2.y, o2.z, __uint_as_float(pix));
      e[1] = make_float4(rd.x, rd.y, rd.z, __uint_as_float(depth + 1));
      e[2] = make_float4(w.x * mat.w, w.y * mat.w, w.z * mat.w, 0.f);
    }
    nR += __popc(mr);
    made_r += __popc(mr);
    if (mode == M_PRIMARY && active) {
      const uint32_t eye = pix >= P;
      const uint32_t pi = pix - eye * P;
      uint32_t* hid = eye ? a.hit_R : a.hit_L;
      float* dep = eye ? a.depth_R : a.depth_L;
      if (hid) hid[pi] = id;
      if (dep) dep[pi] = hit ? t * dot(d, v3(cam.fwd[0], cam.fwd[1], cam.fwd[2])) : INFINITY;
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
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * n3; i += gridDim.x * blockDim.x) {
    const float v = fminf(1.f, (float)acc[i] * inv_scale);
    if (i < n3) out_L[i] = v; else out_R[i - n3] = v;
  }
}

__global__ void k_counts(const uint32_t* counters, uint64_t primary, uint64_t* out) {
  if (threadIdx.x != 0) return;
  out[0] = primary;
  out[1] = counters[C_SHADOW];
  out[2] = counters[C_REFL];
}

template <bool COUNT, bool WIDE>
int blocks_per_sm() {
  static int cached = 0;
  if (!cached) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render<COUNT, WIDE>, kThreads,
                                                  kMaxTopBytes);
    cached = per_sm > 0 ? per_sm : 1;
  }
  return cached;
}

template <bool COUNT, bool WIDE>
cudaError_t render_impl(const RenderArgs& a, Workspace& ws, cudaStream_t st) {
  const uint64_t P = (uint64_t)a.cam.W * a.cam.H;
  KParams kp;
  kp.a = a;
  kp.accum = ws.accum;
  kp.wq = ws.wq;
  kp.counters = ws.counters;
  kp.cap_s = ws.cap_s;
  kp.cap_r = ws.cap_r;
  kp.n_tiles = a.plist ? (a.plist_n + 31u) / 32u
                       : (a.eyes == 3u ? 2u : 1u) * a.cam.tiles_x * a.cam.tiles_y;
  const int grid = render_grid();
  if ((uint64_t)grid * (kThreads / 32) > ws.n_warps) return cudaErrorInvalidValue;
  cudaMemsetAsync(ws.counters, 0, C_TOTAL * sizeof(uint32_t), st);
  // clear the colour sums of the eyes this render traces
  const bool left = !a.plist && (a.eyes & 1u), right = a.plist || (a.eyes & 2u);
  if (left && right) cudaMemsetAsync(ws.accum, 0, 2 * P * 3 * sizeof(uint32_t), st);
  else if (left) cudaMemsetAsync(ws.accum, 0, P * 3 * sizeof(uint32_t), st);
  else cudaMemsetAsync(ws.accum + 3 * P, 0, P * 3 * sizeof(uint32_t), st);
  if (a.work) cudaMemsetAsync(a.work, 0, 9 * sizeof(uint64_t), st);
  profile_mark(ws, ST_CLEAR, st);
  const size_t top_bytes = (WIDE && !COUNT) ? 7 * sizeof(float4) * a.sc.n_top : 0;
  k_render<COUNT, WIDE><<<grid, kThreads, top_bytes, st>>>(kp);
  profile_mark(ws, a.trace_stage, st);
  const uint32_t n3 = (uint32_t)(P * 3);
  if (a.resolve) {
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
  int b = blocks_per_sm<false, true>();
  if (blocks_per_sm<false, false>() > b) b = blocks_per_sm<false, false>();
  if (blocks_per_sm<true, false>() > b) b = blocks_per_sm<true, false>();
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
  if (a.work) return render_impl<true, false>(a, ws, st);
  return a.binary || a.sc.n4 == 0 ? render_impl<false, false>(a, ws, st)
                                   : render_impl<false, true>(a, ws, st);
}

}  // namespace rt
