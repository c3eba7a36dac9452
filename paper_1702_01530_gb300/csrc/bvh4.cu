// 4-wide BVH collapsed from a binary tree (the SAH render tree; sm_103a).
//
// Every internal node of the binary tree at even depth becomes one 4-wide
// node whose children are its grandchildren (a child that is a leaf stays a
// direct leaf child): 2 to 4 children, the same boxes, the same leaves.
// Traversal then needs about half the dependent node fetches per ray and
// tests four boxes per fetch. Nodes whose 4-wide depth is below `top_depth`
// are numbered first (0 .. n_top-1) so the renderer can stage them in shared
// memory; the rest follow in binary-tree index order. The binary tree's root
// is node 0 and `parent` gives the parent of each inner node.
//
// Node layout (7 x float4 = 112 B): lo.x[4], hi.x[4], lo.y[4], hi.y[4],
// lo.z[4], hi.z[4], child[4] (int bits: >= 0 4-wide node, < 0 leaf ~k).
// An unused slot holds child kEmptyChild (never visited: the traversal masks
// it) and the point box (+inf, +inf, +inf).
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_internal.cuh"

namespace rt {
namespace {

__global__ void k_depth_flags(const int32_t* __restrict__ parent, uint32_t n_inner, int top_depth,
                              uint32_t* flag_top, uint32_t* flag_rest, uint8_t* depth_out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_inner) return;
  int d = 0;
  int32_t p = (int32_t)i;
  while (p != 0 && d < 200) { p = parent[p]; ++d; }
  const bool even = (d & 1) == 0;
  const bool top = even && (d >> 1) < top_depth;
  flag_top[i] = top ? 1u : 0u;
  flag_rest[i] = (even && !top) ? 1u : 0u;
  depth_out[i] = (uint8_t)(d < 255 ? d : 255);
}

__device__ __forceinline__ void child_box(const float4* nodes, int32_t node, int slot, float lo[3],
                                          float hi[3]) {
  const float4 a = nodes[4 * (size_t)node + (slot ? 1 : 0)];
  const float4 c = nodes[4 * (size_t)node + 2];
  lo[0] = a.x; hi[0] = a.y; lo[1] = a.z; hi[1] = a.w;
  lo[2] = slot ? c.z : c.x;
  hi[2] = slot ? c.w : c.y;
}

__global__ void k_build4(const float4* __restrict__ nodes, uint32_t n_inner,
                         const uint32_t* __restrict__ scan_top, const uint32_t* __restrict__ scan_rest,
                         const uint32_t* __restrict__ flag_top, const uint32_t* __restrict__ flag_rest,
                         float4* __restrict__ nodes4, uint32_t* counts) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t last = n_inner - 1;
  const uint32_t n_top = scan_top[last] + flag_top[last];
  if (i == 0) {
    counts[0] = n_top;
    counts[1] = n_top + scan_rest[last] + flag_rest[last];
  }
  if (i >= n_inner || !(flag_top[i] | flag_rest[i])) return;
  auto idx4 = [&](int32_t g) -> int32_t {
    return (int32_t)(flag_top[g] ? scan_top[g] : n_top + scan_rest[g]);
  };
  float lo[3][4], hi[3][4];
  int32_t ch[4] = {0, 0, 0, 0};
  int slot = 0;
  const float4 ci = nodes[4 * (size_t)i + 3];
  const int32_t kids[2] = {__float_as_int(ci.x), __float_as_int(ci.y)};
  for (int s = 0; s < 2; ++s) {
    const int32_t c = kids[s];
    float l[3], h[3];
    if (c < 0) {
      child_box(nodes, (int32_t)i, s, l, h);
      for (int a = 0; a < 3; ++a) { lo[a][slot] = l[a]; hi[a][slot] = h[a]; }
      ch[slot++] = c;
    } else {
      const float4 cc = nodes[4 * (size_t)c + 3];
      const int32_t gk[2] = {__float_as_int(cc.x), __float_as_int(cc.y)};
      for (int s2 = 0; s2 < 2; ++s2) {
        child_box(nodes, c, s2, l, h);
        for (int a = 0; a < 3; ++a) { lo[a][slot] = l[a]; hi[a][slot] = h[a]; }
        ch[slot++] = gk[s2] < 0 ? gk[s2] : idx4(gk[s2]);
      }
    }
  }
  for (; slot < 4; ++slot) {
    for (int a = 0; a < 3; ++a) { lo[a][slot] = INFINITY; hi[a][slot] = INFINITY; }
    ch[slot] = kEmptyChild;
  }
  float4* o = nodes4 + 7 * (size_t)idx4((int32_t)i);
  o[0] = make_float4(lo[0][0], lo[0][1], lo[0][2], lo[0][3]);
  o[1] = make_float4(hi[0][0], hi[0][1], hi[0][2], hi[0][3]);
  o[2] = make_float4(lo[1][0], lo[1][1], lo[1][2], lo[1][3]);
  o[3] = make_float4(hi[1][0], hi[1][1], hi[1][2], hi[1][3]);
  o[4] = make_float4(lo[2][0], lo[2][1], lo[2][2], lo[2][3]);
  o[5] = make_float4(hi[2][0], hi[2][1], hi[2][2], hi[2][3]);
  o[6] = make_float4(__int_as_float(ch[0]), __int_as_float(ch[1]), __int_as_float(ch[2]),
                     __int_as_float(ch[3]));
}

// exclusive scan in one block (chunked), as in the radix sort
__global__ void k_scan_excl(uint32_t* a, uint32_t len) {
  __shared__ uint32_t part[1024];
  const uint32_t per = (len + blockDim.x - 1) / blockDim.x;
  const uint32_t b = threadIdx.x * per, e = min(len, b + per);
  uint32_t sum = 0;
  for (uint32_t i = b; i < e; ++i) sum += a[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (uint32_t off = 1; off < blockDim.x; off <<= 1) {
    const uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - sum;
  for (uint32_t i = b; i < e; ++i) { const uint32_t v = a[i]; a[i] = run; run += v; }
}

// parent of every internal node of a binary tree (root 0, its own parent)
__global__ void k_inner_parents(const float4* __restrict__ nodes, uint32_t n_inner, int32_t* parent) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_inner) return;
  if (i == 0) parent[0] = 0;
  const float4 e = nodes[4 * (size_t)i + 3];
  const int32_t cl = __float_as_int(e.x), cr = __float_as_int(e.y);
  if (cl > 0 && (uint32_t)cl < n_inner) parent[cl] = (int32_t)i;
  if (cr > 0 && (uint32_t)cr < n_inner) parent[cr] = (int32_t)i;
}

}  // namespace

cudaError_t inner_parents(const float4* nodes, uint32_t n, int32_t* parent, cudaStream_t st) {
  if (n < 2) return cudaSuccess;
  const uint32_t m = n - 1;
  k_inner_parents<<<(m + 255) / 256, 256, 0, st>>>(nodes, m, parent);
  return cudaGetLastError();
}

size_t bvh4_tmp_bytes(uint32_t n) {
  const size_t m = n > 1 ? n - 1 : 1;
  return 4 * ((m * 4 + 255) & ~size_t(255)) + ((m + 255) & ~size_t(255)) + 1024;
}

cudaError_t build_bvh4(const float4* nodes, const int32_t* parent, uint32_t n, int top_depth,
                       float4* nodes4, uint32_t* counts_dev, void* tmp, cudaStream_t st) {
  if (n < 2) return cudaSuccess;   // a single primitive needs no inner node
  const uint32_t m = n - 1;
  char* t = static_cast<char*>(tmp);
  auto take = [&](size_t bytes) { char* p = t; t += (bytes + 255) & ~size_t(255); return p; };
  uint32_t* flag_top = reinterpret_cast<uint32_t*>(take((size_t)m * 4));
  uint32_t* flag_rest = reinterpret_cast<uint32_t*>(take((size_t)m * 4));
  uint32_t* scan_top = reinterpret_cast<uint32_t*>(take((size_t)m * 4));
  uint32_t* scan_rest = reinterpret_cast<uint32_t*>(take((size_t)m * 4));
  uint8_t* depth = reinterpret_cast<uint8_t*>(take(m));
  const int blocks = (int)((m + 255) / 256);
  k_depth_flags<<<blocks, 256, 0, st>>>(parent, m, top_depth, flag_top, flag_rest, depth);
  cudaMemcpyAsync(scan_top, flag_top, (size_t)m * 4, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(scan_rest, flag_rest, (size_t)m * 4, cudaMemcpyDeviceToDevice, st);
  k_scan_excl<<<1, 1024, 0, st>>>(scan_top, m);
  k_scan_excl<<<1, 1024, 0, st>>>(scan_rest, m);
  k_build4<<<blocks, 256, 0, st>>>(nodes, m, scan_top, scan_rest, flag_top, flag_rest, nodes4, counts_dev);
  return cudaGetLastError();
}

}  // namespace rt
