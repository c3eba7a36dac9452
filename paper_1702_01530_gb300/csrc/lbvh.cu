// Linear BVH build on the GPU (sm_103a).
//
// Table 1 of the paper names BVH trees as the GPU-friendly acceleration
// structure; this is the linear BVH over Morton codes:
//   1. k_centroids / k_bounds : FP64 centroids (triangle ((v0+v1)+v2)/3, every
//      operation correctly rounded, no FMA) and their per-axis min/max.
//   2. k_keys                 : q_a = min(1023, floor((c_a - min_a) /
//      (max_a - min_a) * 1024)) (0 when the extent is 0), morton30 with x at
//      bit 3k+2, y at 3k+1, z at 3k; key = morton30 << 32 | primitive id.
//   3. radix sort             : stable LSD sort on the 30 Morton bits
//      (8-bit digits). Keys start in id order, so the result is sorted by the
//      whole 64-bit key.
//   4. k_karras               : binary radix tree over the sorted keys, one
//      thread per internal node (direction, range end, split by binary
//      search on delta(i, j) = clz(key_i ^ key_j)).
//   5. k_refit                : leaf boxes (triangle min/max; sphere c -/+ r in
//      FP64 rounded outward to FP32), written into the parent's child slot;
//      bottom-up refit with one arrival counter per node (the second thread
//      to arrive merges both children and climbs on).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "rt_internal.cuh"

namespace rt {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;                       // items per thread per tile
constexpr int kTile = kSortThreads * kSortItems;    // 2048 keys per block
constexpr int kRedThreads = 256;

struct Bounds6 { double lo[3], hi[3]; };

__device__ __forceinline__ void load_tri(const float* t, uint32_t i, float v[9]) {
  const float* p = t + 10ull * i;
#pragma unroll
  for (int k = 0; k < 9; ++k) v[k] = p[k];
}

__device__ __forceinline__ void centroid(const float* sph, const float* tri, uint32_t ns,
                                         uint32_t i, double c[3]) {
  if (i < ns) {
    const float* p = sph + 5ull * i;
    c[0] = p[0]; c[1] = p[1]; c[2] = p[2];
  } else {
    float v[9];
    load_tri(tri, i - ns, v);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      c[k] = __ddiv_rn(__dadd_rn(__dadd_rn((double)v[k], (double)v[3 + k]), (double)v[6 + k]), 3.0);
  }
}

// per-block partial min/max of the centroids
__global__ void k_centroid_bounds(const float* sph, const float* tri, uint32_t ns, uint32_t n,
                                  Bounds6* partial) {
  __shared__ double s[6][kRedThreads];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double c[3];
    centroid(sph, tri, ns, i, c);
#pragma unroll
    for (int k = 0; k < 3; ++k) { lo[k] = fmin(lo[k], c[k]); hi[k] = fmax(hi[k], c[k]); }
  }
  for (int k = 0; k < 3; ++k) { s[k][threadIdx.x] = lo[k]; s[3 + k][threadIdx.x] = hi[k]; }
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 3; ++k) {
        s[k][threadIdx.x] = fmin(s[k][threadIdx.x], s[k][threadIdx.x + w]);
        s[3 + k][threadIdx.x] = fmax(s[3 + k][threadIdx.x], s[3 + k][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) { partial[blockIdx.x].lo[k] = s[k][0]; partial[blockIdx.x].hi[k] = s[3 + k][0]; }
}

__global__ void k_reduce_bounds(Bounds6* partial, int nparts) {
  if (threadIdx.x != 0) return;
  Bounds6 b = partial[0];
  for (int p = 1; p < nparts; ++p)
    for (int k = 0; k < 3; ++k) { b.lo[k] = fmin(b.lo[k], partial[p].lo[k]); b.hi[k] = fmax(b.hi[k], partial[p].hi[k]); }
  partial[0] = b;
}

__device__ __forceinline__ uint32_t quantise(double c, double lo, double hi) {
  double ext = __dsub_rn(hi, lo);
  if (ext == 0.0) return 0u;
  double f = floor(__dmul_rn(__ddiv_rn(__dsub_rn(c, lo), ext), 1024.0));
  f = fmin(1023.0, fmax(0.0, f));
  return (uint32_t)f;
}

__device__ __forceinline__ uint32_t spread10(uint32_t x) {  // bit k -> bit 3k
  x &= 0x3FFu;
  x = (x | (x << 16)) & 0x030000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

__global__ void k_keys(const float* sph, const float* tri, uint32_t ns, uint32_t n,
                       const Bounds6* b, uint64_t* keys) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double c[3];
  centroid(sph, tri, ns, i, c);
  uint32_t qx = quantise(c[0], b->lo[0], b->hi[0]);
  uint32_t qy = quantise(c[1], b->lo[1], b->hi[1]);
  uint32_t qz = quantise(c[2], b->lo[2], b->hi[2]);
  uint32_t m = (spread10(qx) << 2) | (spread10(qy) << 1) | spread10(qz);
  keys[i] = ((uint64_t)m << 32) | i;
}

// ---------------------------------------------------------------- radix sort
__global__ void k_hist(const uint64_t* keys, uint32_t n, int shift, uint32_t* ghist, int nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  uint64_t base = (uint64_t)blockIdx.x * kTile;
  for (int r = 0; r < kSortItems; ++r) {
    uint64_t i = base + (uint64_t)r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
  }
  __syncthreads();
  ghist[(size_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of a[0..len) in one block of 1024 threads (chunked)
__global__ void k_scan(uint32_t* a, uint32_t len) {
  __shared__ uint32_t part[1024];
  uint32_t per = (len + blockDim.x - 1) / blockDim.x;
  uint32_t b = threadIdx.x * per, e = min(len, b + per);
  uint32_t sum = 0;
  for (uint32_t i = b; i < e; ++i) sum += a[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (uint32_t off = 1; off < blockDim.x; off <<= 1) {
    uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - sum;
  for (uint32_t i = b; i < e; ++i) { uint32_t v = a[i]; a[i] = run; run += v; }
}

// stable scatter: rounds of 256 consecutive keys; ranks within a warp from
// match masks, across warps from per-warp digit counts in shared memory
__global__ void k_scatter(const uint64_t* in, uint64_t* out, uint32_t n, int shift,
                          const uint32_t* gscan, int nblocks) {
  __shared__ uint32_t base[256];
  __shared__ uint32_t wcnt[kSortThreads / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base[tid] = gscan[(size_t)tid * nblocks + blockIdx.x];
  for (int w = 0; w < kSortThreads / 32; ++w) wcnt[w][tid] = 0;
  __syncthreads();
  uint64_t tile = (uint64_t)blockIdx.x * kTile;
  for (int r = 0; r < kSortItems; ++r) {
    uint64_t i = tile + (uint64_t)r * kSortThreads + tid;
    bool valid = i < n;
    uint64_t key = valid ? in[i] : 0ull;
    uint32_t dig = valid ? (uint32_t)((key >> shift) & 0xFF) : 256u;
    uint32_t peers = __match_any_sync(0xFFFFFFFFu, dig);
    uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[warp][dig] = __popc(peers);
    __syncthreads();
    // thread d: turn the per-warp counts of digit d into exclusive offsets
    {
      uint32_t acc = 0;
      for (int w = 0; w < kSortThreads / 32; ++w) {
        uint32_t c = wcnt[w][tid];
        wcnt[w][tid] = acc;
        acc += c;
      }
      // base[] is advanced after the scatter below (wcnt holds offsets now)
      __syncthreads();
      if (valid) out[base[dig] + wcnt[warp][dig] + rank] = key;
      __syncthreads();
      base[tid] += acc;
      for (int w = 0; w < kSortThreads / 32; ++w) wcnt[w][tid] = 0;
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------ radix tree
__device__ __forceinline__ int delta(const uint64_t* k, int64_t n, int64_t i, int64_t j) {
  if (j < 0 || j >= n) return -1;
  return __clzll(k[i] ^ k[j]);
}

__global__ void k_karras(const uint64_t* keys, uint32_t n, float4* nodes, int32_t* parent) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n - 1) return;
  int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) > 0 ? 1 : -1;
  int dmin = delta(keys, n, i, i - d);
  int64_t lmax = 2;
  while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int64_t l = 0;
  for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
  int64_t j = i + l * d;
  int dnode = delta(keys, n, i, j);
  int64_t s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int64_t g = i + s * d + min(d, 0);
  int32_t left = (min(i, j) == g) ? ~(int32_t)g : (int32_t)g;
  int32_t right = (max(i, j) == g + 1) ? ~(int32_t)(g + 1) : (int32_t)(g + 1);
  nodes[4 * i + 3] = make_float4(__int_as_float(left), __int_as_float(right), 0.f, 0.f);
  parent[left >= 0 ? left : (int64_t)n - 1 + ~left] = (int32_t)i;
  parent[right >= 0 ? right : (int64_t)n - 1 + ~right] = (int32_t)i;
  if (i == 0) parent[0] = -1;
}

// write box (lo, hi) into the child slot `slot` (0 left, 1 right) of node p
__device__ __forceinline__ void store_child_box(float4* nodes, int32_t p, int slot,
                                                const float lo[3], const float hi[3]) {
  float* f = reinterpret_cast<float*>(nodes + 4 * (int64_t)p);
  if (slot == 0) {
    f[0] = lo[0]; f[1] = hi[0]; f[2] = lo[1]; f[3] = hi[1];
    f[8] = lo[2]; f[9] = hi[2];
  } else {
    f[4] = lo[0]; f[5] = hi[0]; f[6] = lo[1]; f[7] = hi[1];
    f[10] = lo[2]; f[11] = hi[2];
  }
}

__global__ void k_refit(const float* sph, const float* tri, uint32_t ns, uint32_t n,
                        const uint64_t* keys, float4* nodes, float4* prims, const int32_t* parent,
                        uint32_t* arrivals, uint32_t* err) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  uint32_t id = (uint32_t)(keys[k] & 0xFFFFFFFFull);
  float lo[3], hi[3];
  if (id < ns) {
    const float* p = sph + 5ull * id;
    float r = p[3];
    uint32_t mat = __float_as_uint(p[4]);
    for (int a = 0; a < 3; ++a) {
      lo[a] = __double2float_rd(__dsub_rd((double)p[a], (double)r));
      hi[a] = __double2float_ru(__dadd_ru((double)p[a], (double)r));
    }
    prims[3ull * k + 0] = make_float4(p[0], p[1], p[2], __uint_as_float(id));
    prims[3ull * k + 1] = make_float4(r, 0.f, 0.f, __uint_as_float(mat));
    prims[3ull * k + 2] = make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    float v[9];
    load_tri(tri, id - ns, v);
    uint32_t mat = __float_as_uint(tri[10ull * (id - ns) + 9]);
    for (int a = 0; a < 3; ++a) {
      lo[a] = fminf(v[a], fminf(v[3 + a], v[6 + a]));
      hi[a] = fmaxf(v[a], fmaxf(v[3 + a], v[6 + a]));
    }
    prims[3ull * k + 0] = make_float4(v[0], v[1], v[2], __uint_as_float(id));
    prims[3ull * k + 1] = make_float4(v[3] - v[0], v[4] - v[1], v[5] - v[2], __uint_as_float(mat));
    prims[3ull * k + 2] = make_float4(v[6] - v[0], v[7] - v[1], v[8] - v[2], 0.f);
  }
  if (n == 1) {  // no internal node: keep the leaf box in the spare slot 0
    store_child_box(nodes, 0, 0, lo, hi);
    return;
  }
  int32_t child = ~(int32_t)k;
  int32_t p = parent[n - 1 + k];
  for (int step = 0; step < 130; ++step) {
    float4 cd = __ldcg(nodes + 4 * (int64_t)p + 3);
    int slot = (__float_as_int(cd.x) == child) ? 0 : 1;
    store_child_box(nodes, p, slot, lo, hi);
    __threadfence();
    if (atomicAdd(&arrivals[p], 1u) == 0u) return;  // sibling not done yet
    __threadfence();
    // both children are in: merge them into the box of p
    float4 a = __ldcg(nodes + 4 * (int64_t)p + 0);
    float4 b = __ldcg(nodes + 4 * (int64_t)p + 1);
    float4 c = __ldcg(nodes + 4 * (int64_t)p + 2);
    lo[0] = fminf(a.x, b.x); hi[0] = fmaxf(a.y, b.y);
    lo[1] = fminf(a.z, b.z); hi[1] = fmaxf(a.w, b.w);
    lo[2] = fminf(c.x, c.z); hi[2] = fmaxf(c.y, c.w);
    if (p == 0) return;                              // root reached
    child = p;
    p = parent[p];
  }
  atomicOr(err, ERR_BUILD);
}

}  // namespace

size_t lbvh_tmp_bytes(uint32_t n) {
  size_t nblocks = (n + kTile - 1) / kTile;
  size_t red_blocks = 256;
  size_t b = 0;
  b += 256 * sizeof(Bounds6) + red_blocks * sizeof(Bounds6);  // bounds
  b += (size_t)n * 8 + 256;                                  // ping-pong keys
  b += 256 * nblocks * 4 + 256;                              // histogram
  b += (size_t)n * 4 + 256;                                  // arrival counters
  return b + 1024;
}

cudaError_t build_lbvh(const float4* d_sph_in, const float* d_tri_in, uint32_t ns, uint32_t nt,
                       float4* d_nodes, float4* d_prims, uint64_t* d_keys, int32_t* d_parent,
                       void* d_tmp, size_t tmp_bytes, uint32_t* d_err, cudaStream_t st) {
  const float* sph = reinterpret_cast<const float*>(d_sph_in);
  uint32_t n = ns + nt;
  if (tmp_bytes < lbvh_tmp_bytes(n)) return cudaErrorInvalidValue;
  int nblocks = (int)((n + kTile - 1) / kTile);
  char* t = reinterpret_cast<char*>(d_tmp);
  auto take = [&](size_t bytes) { char* p = t; t += (bytes + 255) & ~size_t(255); return p; };
  Bounds6* partial = reinterpret_cast<Bounds6*>(take(256 * sizeof(Bounds6)));
  uint64_t* keys_b = reinterpret_cast<uint64_t*>(take((size_t)n * 8));
  uint32_t* hist = reinterpret_cast<uint32_t*>(take(256ull * nblocks * 4));
  uint32_t* arrivals = reinterpret_cast<uint32_t*>(take((size_t)n * 4));

  int red_grid = (int)std::min<uint32_t>(256u, (n + kRedThreads - 1) / kRedThreads);
  k_centroid_bounds<<<red_grid, kRedThreads, 0, st>>>(sph, d_tri_in, ns, n, partial);
  k_reduce_bounds<<<1, 32, 0, st>>>(partial, red_grid);
  k_keys<<<(n + 255) / 256, 256, 0, st>>>(sph, d_tri_in, ns, n, partial, d_keys);
  uint64_t* a = d_keys;
  uint64_t* b = keys_b;
  for (int shift = 32; shift < 64; shift += 8) {
    k_hist<<<nblocks, kSortThreads, 0, st>>>(a, n, shift, hist, nblocks);
    k_scan<<<1, 1024, 0, st>>>(hist, 256u * nblocks);
    k_scatter<<<nblocks, kSortThreads, 0, st>>>(a, b, n, shift, hist, nblocks);
    uint64_t* x = a; a = b; b = x;
  }
  // four passes: the sorted keys are back in d_keys
  if (n > 1) {
    k_karras<<<(n - 1 + 255) / 256, 256, 0, st>>>(d_keys, n, d_nodes, d_parent);
    cudaMemsetAsync(arrivals, 0, (size_t)n * 4, st);
  } else {
    cudaMemsetAsync(d_parent, 0xFF, 4, st);
  }
  k_refit<<<(n + 255) / 256, 256, 0, st>>>(sph, d_tri_in, ns, n, d_keys, d_nodes, d_prims,
                                           d_parent, arrivals, d_err);
  return cudaGetLastError();
}

}  // namespace rt
