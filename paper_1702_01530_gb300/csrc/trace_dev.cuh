// Device-side tracing primitives shared by the single-pair renderer
// (trace.cu) and the batched renderer (batch.cu): compile-time knobs, vector
// helpers, the ray-sphere and Moller-Trumbore tests, the BVH traversals and
// the fixed-point colour accumulation. Everything sits in an anonymous
// namespace, so each translation unit owns its copy.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_internal.cuh"

namespace rt {
namespace {

// Tuning knobs (compile-time; times are means of 100 1080p blob pairs on
// GB300, SAH tree, both eyes of a 4x4-pixel tile per warp: 1.042 ms by
// default, 0.221 ms for a 10-primitive scene):
// RT_MIN_BLOCKS = minimum resident blocks per SM requested from the register
// allocator (0 = no request; 9 measured best: the default walk fits 56
// registers without spills, 36 warps per SM; against 8 blocks (64 registers,
// 32 warps) 1.005 against 1.014 ms per 1080p blob pair and 13.94 against
// 14.05 ms per 4K terrain frame; 6 blocks: 1.051 / 0.216 ms; 7 blocks: 1.048
// ms; 10 blocks (48 registers, spills in the shading code): 1.047 / 0.242 ms
// in earlier builds); RT_WHILE_WHILE = 1 postpones the first leaf a ray
// meets and keeps descending until every active lane of the warp holds a
// leaf, so the leaf tests of a warp run together instead of interleaving
// with node visits (the "while-while" loop of Aila & Laine, HPG 2009) --
// 1.247 ms with one primitive per leaf, hence off by default.
#ifndef RT_MIN_BLOCKS
#define RT_MIN_BLOCKS 9
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
// binary traversal keeps the top of its stack in a register: a pop hands
// the register over at once and reloads it from local memory in the
// background, so the pop and the next node fetch do not wait in series;
// 1.093 ms: off by default
#ifndef RT_STACK_TOP_REG
#define RT_STACK_TOP_REG 0
#endif
// binary traversal prefetches both children of every visited node into L1
// (prefetch.global.L1) as soon as their indices are known, so a child's
// fetch that misses L1 overlaps the current node's slab tests; 1.583
// against 1.299 ms (LBVH, one eye per warp): off
#ifndef RT_PREFETCH
#define RT_PREFETCH 0
#endif
// binary traversal defers leaf tests: a lane keeps up to two leaves pending
// and walks on; the warp tests the pending leaves together once
// RT_DEFER_LEAVES lanes hold one, or as soon as any lane can go no further
// (both slots full and the next node a leaf, or nothing left to visit).
// Same images; 1.302 ms at 16 lanes against 1.042 (1.399 / 1.417 / 1.442 at
// 16 / 8 / 4 against 1.149 with one eye per warp), so 0 = off by default
#ifndef RT_DEFER_LEAVES
#define RT_DEFER_LEAVES 0
#endif
// binary traversal reads a 64-byte node with two 32-byte loads
// (ld.global.nc.v8.f32, sm_100 and later) instead of four 16-byte ones:
// half the load instructions and L1 requests per node visit; 1 = plain,
// 2 = with an L1 evict-last hint. 1.149 / 1.150 ms against 1.146 (SAH
// tree, one eye per warp): off by default
#ifndef RT_LD256
#define RT_LD256 0
#endif
// 4-wide closest-hit traversal pushes the other hit children farthest first
#ifndef RT_ORDERED_PUSH
#define RT_ORDERED_PUSH 0
#endif
// RT_FAST_RCP = 1: ray reciprocals and the triangle determinant's reciprocal
// by the approximate hardware reciprocal (rcp.approx.f32, at most 1 ulp off)
// instead of the correctly rounded one (whose slow path also cost the render
// kernel 24 bytes of register spills), the robust slab factor widened to
// match, and pixel positions by multiplication with host-computed scales
// instead of two divisions per primary ray: 1.050 -> 1.020 ms per 1080p blob
// pair, 0.222 -> 0.214 ms for the 10-primitive scene; on by default
#ifndef RT_FAST_RCP
#define RT_FAST_RCP 1
#endif
// RT_PRIMARY_STORE = 1: a pixel's primary ray stores its contribution
// (store_first) and the colour sums are not cleared before a render; 0: every
// contribution is an atomic add onto sums cleared by a memset. Same images;
// 1.018 -> 1.012 ms per 1080p blob pair, 0.212 -> 0.182 ms for the
// 10-primitive scene at 1080p.
#ifndef RT_PRIMARY_STORE
#define RT_PRIMARY_STORE 1
#endif
constexpr int kThreads = 128;
// conservative slab exit (Ize 2013): 1 + 2 gamma_3 with correctly rounded
// reciprocals, 1 + 2 gamma_5 when each may be one ulp off
constexpr float kRobust = RT_FAST_RCP ? 1.0000006f : 1.00000036f;

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

__device__ __forceinline__ float rcp_f(float x) {
#if RT_FAST_RCP
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#else
  return __frcp_rn(x);
#endif
}

__device__ __forceinline__ float safe_rcp(float x) {
  const float tiny = 8.271806e-25f;  // 2^-80
  return rcp_f(fabsf(x) > tiny ? x : copysignf(tiny, x));
}

struct WorkCount { uint32_t inner, sphere, tri; };

// Two float4 of one 32-byte aligned block through the read-only path in one
// 256-bit load.
__device__ __forceinline__ void ldg2x16(const float4* p, float4& u, float4& v) {
#if RT_LD256 == 2
  asm("ld.global.nc.L1::evict_last.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
#else
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
#endif
      : "=f"(u.x), "=f"(u.y), "=f"(u.z), "=f"(u.w), "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p));
}

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
  float inv = rcp_f(det);
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
    if (node >= 0) {
      // the iteration bound is checked on node visits only: a leaf visit
      // pushes nothing, so a run of them ends with the (bounded) stack
      if (it >= it_max || (uint32_t)node >= n - 1) {
        atomicOr(err, it >= it_max ? ERR_ITER : ERR_INDEX);
        break;
      }
      const float4* np = sc.nodes + 4 * (size_t)node;
      float4 a, b, c, e;
      if (RT_LD256) {                  // nodes are 64-byte aligned
        ldg2x16(np, a, b);
        ldg2x16(np + 2, c, e);
      } else {
        a = __ldg(np); b = __ldg(np + 1); c = __ldg(np + 2); e = __ldg(np + 3);
      }
      if (COUNT) wc.inner++;
      if (RT_PREFETCH) {
        const int32_t pl = __float_as_int(e.x), pr = __float_as_int(e.y);
        // only in-range children are prefetched (the traversal checks them again)
        if (pl >= 0 ? (uint32_t)pl < n - 1 : (uint32_t)~pl < n)
          asm volatile("prefetch.global.L1 [%0];" ::"l"(pl >= 0 ? sc.nodes + 4 * (size_t)pl
                                                                 : sc.prims + 3 * (size_t)~pl));
        if (pr >= 0 ? (uint32_t)pr < n - 1 : (uint32_t)~pr < n)
          asm volatile("prefetch.global.L1 [%0];" ::"l"(pr >= 0 ? sc.nodes + 4 * (size_t)pr
                                                                 : sc.prims + 3 * (size_t)~pr));
      }
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

#if RT_DEFER_LEAVES
// Binary traversal with deferred leaves (the speculative "while-while" idea
// of Aila & Laine, HPG 2009, in one loop): node visits and leaf tests of a
// warp run in separate passes of the same iteration, so a leaf met by one
// lane no longer costs every other lane a full primitive test. A deferred
// leaf can only make the closest-hit bound tcur shrink later, so the set of
// leaves tested contains the one the eager walk would accept: the hit (t,
// lower id on ties) and the any-hit answer are the same.
template <bool ANY>
__device__ __forceinline__ bool traverse_dl(const DeviceScene& sc, V3 o, V3 d, float tmax,
                                            float& t_best, uint32_t& id_best, uint32_t& k_best,
                                            uint32_t* err) {
  constexpr int32_t kDone = 0x7FFFFFFF;        // larger than any internal node index
  const V3 idir = v3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
  const V3 ood = v3(o.x * idir.x, o.y * idir.y, o.z * idir.z);
  int32_t stack[kStackSize];
  int sp = 0;
  const uint32_t n = sc.n_prims;
  int32_t node = n == 1 ? ~0 : 0;
  int32_t l0 = 0, l1 = 0;                      // pending leaves (~k), 0 = empty; l1 != 0 => l0 != 0
  // every iteration visits a node, moves a leaf to a slot or tests the
  // slots, and a ray visits each node and leaf at most once
  const uint32_t it_max = 2u * n + 64u;
  float tcur = ANY ? tmax : t_best;
  bool any = false;
  for (uint32_t it = 0;; ++it) {
    if (it >= it_max) { atomicOr(err, ERR_ITER); break; }
    if (node >= 0 && node != kDone) {
      if ((uint32_t)node >= n - 1) { atomicOr(err, ERR_INDEX); break; }
      const float4* np = sc.nodes + 4 * (size_t)node;
      const float4 a = __ldg(np), b = __ldg(np + 1), c = __ldg(np + 2), e = __ldg(np + 3);
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
        if (sp >= kStackSize) { atomicOr(err, ERR_STACK); break; }
        const bool swap = in1 < in0;
        stack[sp++] = swap ? cl : cr;
        node = swap ? cr : cl;
      } else if (hit0 | hit1) {
        node = hit0 ? cl : cr;
      } else {
        node = sp ? stack[--sp] : kDone;
      }
    }
    if (node < 0 && l0 == 0) { l0 = node; node = sp ? stack[--sp] : kDone; }
    if (node < 0 && l1 == 0) { l1 = node; node = sp ? stack[--sp] : kDone; }
    const bool pend = l0 != 0;
    const bool stuck = pend && (node < 0 || node == kDone);
    const unsigned m = __activemask();
    const bool flush = __any_sync(m, stuck) || __popc(__ballot_sync(m, pend)) >= RT_DEFER_LEAVES;
    if (flush && pend) {
      bool bad = false;
#pragma unroll 1
      for (int s = 0; s < 2; ++s) {
        const int32_t lf = s ? l1 : l0;
        if (lf == 0) break;
        const uint32_t k = (uint32_t)~lf;
        if (k >= n) { bad = true; break; }
        const float4* pp = sc.prims + 3 * (size_t)k;
        const float4 p0 = __ldg(pp), p1 = __ldg(pp + 1);
        const uint32_t id = __float_as_uint(p0.w);
        float t;
        const bool h = id < sc.n_spheres ? hit_sphere(p0, p1.x, o, d, t)
                                         : hit_tri(p0, p1, __ldg(pp + 2), o, d, t);
        if (ANY) {
          if (h && t < tmax) { any = true; node = kDone; break; }
        } else if (h && (t < tcur || (t == tcur && id < id_best))) {
          tcur = t;
          id_best = id;
          k_best = k;
          any = true;
        }
      }
      if (bad) { atomicOr(err, ERR_INDEX); break; }
      l0 = l1 = 0;
    }
    if (node == kDone && l0 == 0) break;
  }
  if (!ANY) t_best = tcur;
  return any;
}
#endif

// The instrumented (COUNT) walk and the binary renders use the binary tree
// in sc.nodes (the SAH tree, or the LBVH whose node visits define the
// algorithmic work); a 4-wide render walks the 4-wide tree (the same leaves,
// the same hits).
// TREE: kTreeBinary (sc.nodes) or kTreeWide4 (sc.nodes4 = the 4-wide tree)
template <bool ANY, bool COUNT, int TREE>
__device__ __forceinline__ bool trace_ray(const DeviceScene& sc, const float4* top, V3 o, V3 d,
                                          float tmax, float& t_best, uint32_t& id_best,
                                          uint32_t& k_best, WorkCount& wc, uint32_t* err) {
  if (TREE == kTreeWide4 && !COUNT) return traverse4<ANY>(sc, top, o, d, tmax, t_best, id_best, k_best, err);
#if RT_DEFER_LEAVES
  if (!COUNT) return traverse_dl<ANY>(sc, o, d, tmax, t_best, id_best, k_best, err);
#endif
#if RT_WHILE_WHILE
  return traverse_ww<ANY, COUNT>(sc, o, d, tmax, t_best, id_best, k_best, wc, err);
#else
  return traverse<ANY, COUNT>(sc, o, d, tmax, t_best, id_best, k_best, wc, err);
#endif
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// Primary ray of pixel (px, py) of one eye (0 = left, 1 = right): both eyes
// aim at the same point Q of the window on the convergence plane.
__device__ __forceinline__ void primary_ray(const CameraParams& cam, uint32_t px, uint32_t py,
                                            uint32_t eye, V3& o, V3& d) {
#if RT_FAST_RCP
  const float nx = fmaf((float)px + 0.5f, cam.sx, -cam.tan_x);
  const float ny = fmaf(-((float)py + 0.5f), cam.sy, cam.tan_y);
#else
  const float nx = (2.f * ((float)px + 0.5f) / (float)cam.W - 1.f) * cam.tan_x;
  const float ny = (1.f - 2.f * ((float)py + 0.5f) / (float)cam.H) * cam.tan_y;
#endif
  const V3 E = v3(cam.eye[0], cam.eye[1], cam.eye[2]);
  const V3 Rt = v3(cam.right[0], cam.right[1], cam.right[2]);
  const V3 U = v3(cam.up[0], cam.up[1], cam.up[2]);
  const V3 F = v3(cam.fwd[0], cam.fwd[1], cam.fwd[2]);
  const V3 Q = E + (F + Rt * nx + U * ny) * cam.zc;
  o = E + Rt * (eye ? cam.half_sep : -cam.half_sep);
  d = normalize(Q - o);
}

// Surface at the closest hit (primitive slot k, id): hit point, geometric
// normal turned against the ray, material, and the secondary-ray offset
// eps = 1e-4 max(1, |p|_inf).
__device__ __forceinline__ void hit_surface(const float4* prims, const float4* mats,
                                            uint32_t n_spheres, uint32_t n_mats, uint32_t k,
                                            uint32_t id, V3 o, V3 d, float t, uint32_t* err, V3& p,
                                            V3& nrm, float4& mat, float& eps) {
  const float4* pp = prims + 3 * (size_t)k;
  const float4 p0 = __ldg(pp), p1 = __ldg(pp + 1);
  p = o + d * t;
  uint32_t mid = __float_as_uint(p1.w);
  if (id < n_spheres) nrm = (p - xyz(p0)) * (1.f / p1.x);
  else nrm = normalize(cross(xyz(p1), xyz(__ldg(pp + 2))));
  if (dot(nrm, d) > 0.f) nrm = nrm * -1.f;
  if (mid >= n_mats) { atomicOr(err, ERR_INDEX); mid = 0; }
  mat = __ldg(mats + mid);
  eps = 1e-4f * fmaxf(1.f, fmax3(fabsf(p.x), fabsf(p.y), fabsf(p.z)));
}

// Shadow ray from o2 towards light lp: unit direction lh, distance ld, and
// n.l scaled by the light's intensity and (1 - reflectivity); returns
// whether the light faces the surface (n.l > 0).
__device__ __forceinline__ bool light_ray(float4 lp, V3 o2, V3 nrm, float refl, V3& lh, float& ld,
                                          float& ndl) {
  const V3 lv = xyz(lp) - o2;
  const float inv = rsqrtf(dot(lv, lv));
  ld = dot(lv, lv) * inv;
  lh = lv * inv;
  ndl = dot(nrm, lh);
  const bool emit = ndl > 0.f;
  ndl *= lp.w * (1.f - refl);
  return emit;
}

// Mirror direction of d about nrm, renormalised.
__device__ __forceinline__ V3 mirror_dir(V3 d, V3 nrm) {
  return normalize(d - nrm * (2.f * dot(d, nrm)));
}

__device__ __forceinline__ void accumulate(uint32_t* acc, uint32_t pix, float r, float g, float b,
                                           float scale) {
  uint32_t* p = acc + 3 * (size_t)pix;
  atomicAdd(p + 0, __float2uint_rn(r * scale));
  atomicAdd(p + 1, __float2uint_rn(g * scale));
  atomicAdd(p + 2, __float2uint_rn(b * scale));
}

// The first contribution to a pixel: its primary ray's, stored rather than
// added, so the sums need no clearing before the launch. Every later
// contribution (shadow and mirror rays, all spawned by this ray after this
// store, on this lane or handed on through a release store) is an atomic add
// that the hand-over orders after it.
__device__ __forceinline__ void store_first(uint32_t* acc, uint32_t pix, float r, float g, float b,
                                            float scale) {
  uint32_t* p = acc + 3 * (size_t)pix;
  p[0] = __float2uint_rn(r * scale);
  p[1] = __float2uint_rn(g * scale);
  p[2] = __float2uint_rn(b * scale);
}

}  // namespace
}  // namespace rt
