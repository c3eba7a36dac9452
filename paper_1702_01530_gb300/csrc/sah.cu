// Binned-SAH rebuild of the binary tree over the LBVH's leaves (GPU, sm_103a).
//
// Table 1 of the paper names BVH trees as the acceleration structure and
// leaves the build open. The Morton LBVH (lbvh.cu) is the tree whose topology
// the tests pin bit for bit and whose traversal defines the algorithmic work;
// its splits follow Morton-code bits, not the geometry, so its boxes overlap
// more than they need to. Renders walk a second binary tree over the same
// leaves (one primitive per leaf, the same primitive slots and leaf boxes),
// built top down with the surface area heuristic over binned centroids
// (MacDonald & Booth 1990; binning after Wald 2007): on the 1080p blob pair
// it takes 15 % fewer node visits for shadow and mirror rays and renders the
// same image 11 % faster. Any binary tree over the same conservative leaf
// boxes yields the same closest hit and the same any-hit answer.
//
// One level of the tree per launch, one block per node of the level:
//   1. centroid bounds of the node's leaves (block reduction);
//   2. kBins bins per axis: leaf count and the union of the leaf boxes
//      (shared-memory atomics on order-preserving integer images of floats,
//      one set of bins per warp, merged);
//   3. the split of least SAH cost, area(L) n(L) + area(R) n(R), over the
//      3 (kBins - 1) bin boundaries; an object-median split when the centroids
//      coincide or the depth budget is low, so that no leaf lies deeper than
//      kMaxDepth (the traversal stack holds 64 entries);
//   4. a stable partition of the node's leaf slots (block prefix sums), so
//      the tree does not depend on thread timing;
//   5. the node record: both child boxes, leaf children as ~slot, inner
//      children filled in by the children themselves one level later.
// Node numbering: a binary tree over n leaves has n - 1 inner nodes and each
// owns one split position s (left = [begin, s), right = [s, end)), s in
// [1, n-1]; node id = s - 1, except that the root is 0 and the node whose
// split position is 1 takes the root's id. Ids are therefore unique, dense
// and independent of launch order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_internal.cuh"

namespace rt {
namespace {

#ifndef RT_SAH_THREADS
#define RT_SAH_THREADS 256
#endif
// threads per node (block): 256 measured best (blob scene 12.2 ms, 10M-triangle terrain 485 ms
// for the whole tree; 512: 15.0 / 531 ms, 1024: 22.8 / 778 ms -- the many small nodes of the
// lower levels pay for every thread of their block)
constexpr int kSahThreads = RT_SAH_THREADS;
constexpr int kSahWarps = kSahThreads / 32;
constexpr int kBins = 16;
constexpr int kMaxDepth = 60;        // median splits keep every leaf at or above this depth

struct Job {
  uint32_t begin, end;               // leaf slots idx[begin, end) of this node (end - begin >= 2)
  uint32_t parent_slot;              // parent id << 1 | child slot, or 0xFFFFFFFF for the root
  uint32_t depth;
};

__device__ __forceinline__ int f2o(float f) {        // order-preserving int image of a float
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float o2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

__device__ __forceinline__ float half_area(const float lo[3], const float hi[3]) {
  const float dx = fmaxf(hi[0] - lo[0], 0.f), dy = fmaxf(hi[1] - lo[1], 0.f),
              dz = fmaxf(hi[2] - lo[2], 0.f);
  return dx * dy + dy * dz + dz * dx;
}

// leaf box of slot k: the child box of k's parent that holds leaf ~k
__global__ void k_leaf_boxes(const float4* __restrict__ nodes, const int32_t* __restrict__ parent,
                             uint32_t n, float4* __restrict__ lo, float4* __restrict__ hi) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int32_t p = parent[n - 1 + k];
  const float4 a = nodes[4 * (size_t)p], b = nodes[4 * (size_t)p + 1],
               c = nodes[4 * (size_t)p + 2], e = nodes[4 * (size_t)p + 3];
  if (__float_as_int(e.x) == ~(int32_t)k) {
    lo[k] = make_float4(a.x, a.z, c.x, 0.f);
    hi[k] = make_float4(a.y, a.w, c.y, 0.f);
  } else {
    lo[k] = make_float4(b.x, b.z, c.z, 0.f);
    hi[k] = make_float4(b.y, b.w, c.w, 0.f);
  }
}

__global__ void k_iota(uint32_t* idx, uint32_t n) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) idx[k] = k;
}

__global__ void __launch_bounds__(kSahThreads)
k_sah_level(const float4* __restrict__ leaf_lo, const float4* __restrict__ leaf_hi,
            const uint32_t* __restrict__ idx_in, uint32_t* __restrict__ idx_out,
            const Job* __restrict__ jobs, uint32_t n_jobs, Job* __restrict__ next,
            uint32_t* __restrict__ next_count, float4* __restrict__ out, uint32_t* __restrict__ root_split,
            uint32_t n, uint32_t* __restrict__ err) {
  // bins per warp (fewer shared-memory atomics on one address), merged into warp 0's
  __shared__ int s_cnt[kSahWarps][3][kBins];
  __shared__ int s_box[kSahWarps][3][kBins][6];   // lo xyz, hi xyz as order-preserving ints
  __shared__ int s_red[12];                  // centroid bounds, then child boxes of a median split
  __shared__ uint32_t s_scan[kSahThreads / 32];
  __shared__ float s_cost[3 * (kBins - 1)];
  __shared__ int s_choice[2];                // axis (-1: median), bin
  if (blockIdx.x >= n_jobs) return;
  const Job job = jobs[blockIdx.x];
  const uint32_t b = job.begin, e = job.end, m = e - b;
  const uint32_t tid = threadIdx.x;

  // 1. centroid bounds
  if (tid < 6) s_red[tid] = tid < 3 ? f2o(INFINITY) : f2o(-INFINITY);
  for (int i = tid; i < kSahWarps * 3 * kBins; i += kSahThreads) {
    const int w = i / (3 * kBins), a = (i / kBins) % 3, q = i % kBins;
    s_cnt[w][a][q] = 0;
    for (int c = 0; c < 6; ++c) s_box[w][a][q][c] = c < 3 ? f2o(INFINITY) : f2o(-INFINITY);
  }
  __syncthreads();
  float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (uint32_t i = b + tid; i < e; i += kSahThreads) {
    const uint32_t k = idx_in[i];
    const float4 lo = leaf_lo[k], hi = leaf_hi[k];
    const float c[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
    for (int a = 0; a < 3; ++a) { clo[a] = fminf(clo[a], c[a]); chi[a] = fmaxf(chi[a], c[a]); }
  }
  for (int a = 0; a < 3; ++a) { atomicMin(&s_red[a], f2o(clo[a])); atomicMax(&s_red[3 + a], f2o(chi[a])); }
  __syncthreads();
  float cmin[3], cext[3];
  bool spread = false;
  for (int a = 0; a < 3; ++a) {
    cmin[a] = o2f(s_red[a]);
    cext[a] = o2f(s_red[3 + a]) - cmin[a];
    spread |= cext[a] > 0.f;
  }
  // depth budget: a median split keeps the subtree ceil(log2 m) deep
  const uint32_t lg = 32 - __clz(m - 1);
  const bool median = !spread || job.depth + lg >= (uint32_t)kMaxDepth - 4;

  // 2-3. bins and the SAH split
  if (!median) {
    for (uint32_t i = b + tid; i < e; i += kSahThreads) {
      const uint32_t k = idx_in[i];
      const float4 lo = leaf_lo[k], hi = leaf_hi[k];
      const float c[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
      const float l3[3] = {lo.x, lo.y, lo.z}, h3[3] = {hi.x, hi.y, hi.z};
      for (int a = 0; a < 3; ++a) {
        if (!(cext[a] > 0.f)) continue;
        const int bin = min(kBins - 1, (int)((c[a] - cmin[a]) * ((float)kBins / cext[a])));
        const int w = tid >> 5;
        atomicAdd(&s_cnt[w][a][bin], 1);
        for (int q = 0; q < 3; ++q) {
          atomicMin(&s_box[w][a][bin][q], f2o(l3[q]));
          atomicMax(&s_box[w][a][bin][3 + q], f2o(h3[q]));
        }
      }
    }
    __syncthreads();
    // merge the warps' bins into warp 0's
    for (int i = tid; i < 3 * kBins * 7; i += kSahThreads) {
      const int a = i / (kBins * 7), q = (i / 7) % kBins, f = i % 7;
      if (f == 6) {
        int t = 0;
        for (int w = 0; w < kSahWarps; ++w) t += s_cnt[w][a][q];
        s_cnt[0][a][q] = t;
      } else {
        int v = s_box[0][a][q][f];
        for (int w = 1; w < kSahWarps; ++w) v = f < 3 ? min(v, s_box[w][a][q][f]) : max(v, s_box[w][a][q][f]);
        s_box[0][a][q][f] = v;
      }
    }
    __syncthreads();
    if (tid < 3 * (kBins - 1)) {
      const int a = tid / (kBins - 1), s = tid % (kBins - 1);   // split after bin s
      float llo[3] = {INFINITY, INFINITY, INFINITY}, lhi[3] = {-INFINITY, -INFINITY, -INFINITY};
      float rlo[3] = {INFINITY, INFINITY, INFINITY}, rhi[3] = {-INFINITY, -INFINITY, -INFINITY};
      int nl = 0, nr = 0;
      for (int q = 0; q < kBins; ++q) {
        const int c = s_cnt[0][a][q];
        if (!c) continue;
        float* blo = q <= s ? llo : rlo;
        float* bhi = q <= s ? lhi : rhi;
        for (int x = 0; x < 3; ++x) {
          blo[x] = fminf(blo[x], o2f(s_box[0][a][q][x]));
          bhi[x] = fmaxf(bhi[x], o2f(s_box[0][a][q][3 + x]));
        }
        if (q <= s) nl += c; else nr += c;
      }
      s_cost[tid] = (cext[a] > 0.f && nl > 0 && nr > 0)
                        ? half_area(llo, lhi) * (float)nl + half_area(rlo, rhi) * (float)nr
                        : INFINITY;
    }
    __syncthreads();
    if (tid == 0) {
      int best = -1;
      float bc = INFINITY;
      for (int i = 0; i < 3 * (kBins - 1); ++i)
        if (s_cost[i] < bc) { bc = s_cost[i]; best = i; }   // first of equal costs: deterministic
      s_choice[0] = best < 0 ? -1 : best / (kBins - 1);
      s_choice[1] = best < 0 ? 0 : best % (kBins - 1);
    }
  } else if (tid == 0) {
    s_choice[0] = -1;
    s_choice[1] = 0;
  }
  __syncthreads();
  const int axis = s_choice[0], split_bin = s_choice[1];

  // 4. stable partition into idx_out[b, e): left leaves first, in their order
  uint32_t n_left;
  if (axis < 0) {
    n_left = m / 2;                                  // object median in the current order
    for (uint32_t i = b + tid; i < e; i += kSahThreads) idx_out[i] = idx_in[i];
  } else {
    const float scale = (float)kBins / cext[axis];
    uint32_t cnt_left = 0;
    for (uint32_t base = b; base < e; base += kSahThreads) {
      const uint32_t i = base + tid;
      bool left = false;
      uint32_t k = 0;
      if (i < e) {
        k = idx_in[i];
        const float4 lo = leaf_lo[k], hi = leaf_hi[k];
        const float c = 0.5f * ((&lo.x)[axis] + (&hi.x)[axis]);
        left = min(kBins - 1, (int)((c - cmin[axis]) * scale)) <= split_bin;
      }
      // block-wide exclusive scan of `left`
      const uint32_t ball = __ballot_sync(0xFFFFFFFFu, left);
      const uint32_t lane = tid & 31, warp = tid >> 5;
      __syncthreads();
      if (lane == 0) s_scan[warp] = __popc(ball);
      __syncthreads();
      uint32_t before = 0, chunk = 0;
      for (uint32_t w = 0; w < kSahThreads / 32; ++w) {
        if (w < warp) before += s_scan[w];
        chunk += s_scan[w];
      }
      const uint32_t rank = before + __popc(ball & ((1u << lane) - 1u));
      if (i < e) {
        // lefts from the front in order; rights from the back, reversed
        // (right number r of the range goes to e - 1 - r)
        if (left) idx_out[b + cnt_left + rank] = k;
        else idx_out[e - 1 - ((i - b) - (cnt_left + rank))] = k;
      }
      cnt_left += chunk;
    }
    n_left = cnt_left;
    // the right side was written from the end backwards (reversed); restore
    // its original order so the partition is stable
    __syncthreads();
    const uint32_t n_right = m - n_left;
    for (uint32_t i = tid; i < n_right / 2; i += kSahThreads) {
      const uint32_t x = b + n_left + i, y = e - 1 - i;
      const uint32_t t = idx_out[x];
      idx_out[x] = idx_out[y];
      idx_out[y] = t;
    }
  }
  __syncthreads();
  bool to_median = false;
  if (axis >= 0 && (n_left == 0 || n_left == m)) {
    // cannot happen (the partition repeats the binning arithmetic); an empty
    // side would break the tree, so fall back to the object median
    to_median = true;
    n_left = m / 2;
    for (uint32_t i = b + tid; i < e; i += kSahThreads) idx_out[i] = idx_in[i];
    __syncthreads();
  }

  // child boxes
  float cl[2][3], ch[2][3];
  if (axis >= 0 && !to_median) {
    for (int c = 0; c < 2; ++c)
      for (int x = 0; x < 3; ++x) { cl[c][x] = INFINITY; ch[c][x] = -INFINITY; }
    for (int q = 0; q < kBins; ++q) {
      if (!s_cnt[0][axis][q]) continue;
      const int c = q <= split_bin ? 0 : 1;
      for (int x = 0; x < 3; ++x) {
        cl[c][x] = fminf(cl[c][x], o2f(s_box[0][axis][q][x]));
        ch[c][x] = fmaxf(ch[c][x], o2f(s_box[0][axis][q][3 + x]));
      }
    }
  } else {
    if (tid < 12) s_red[tid] = (tid % 6) < 3 ? f2o(INFINITY) : f2o(-INFINITY);
    __syncthreads();
    float l[2][3], h[2][3];
    for (int c = 0; c < 2; ++c)
      for (int x = 0; x < 3; ++x) { l[c][x] = INFINITY; h[c][x] = -INFINITY; }
    for (uint32_t i = b + tid; i < e; i += kSahThreads) {
      const uint32_t k = idx_out[i];
      const int c = (i - b) < n_left ? 0 : 1;
      const float4 lo = leaf_lo[k], hi = leaf_hi[k];
      l[c][0] = fminf(l[c][0], lo.x); l[c][1] = fminf(l[c][1], lo.y); l[c][2] = fminf(l[c][2], lo.z);
      h[c][0] = fmaxf(h[c][0], hi.x); h[c][1] = fmaxf(h[c][1], hi.y); h[c][2] = fmaxf(h[c][2], hi.z);
    }
    for (int c = 0; c < 2; ++c)
      for (int x = 0; x < 3; ++x) {
        atomicMin(&s_red[6 * c + x], f2o(l[c][x]));
        atomicMax(&s_red[6 * c + 3 + x], f2o(h[c][x]));
      }
    __syncthreads();
    for (int c = 0; c < 2; ++c)
      for (int x = 0; x < 3; ++x) { cl[c][x] = o2f(s_red[6 * c + x]); ch[c][x] = o2f(s_red[6 * c + 3 + x]); }
  }

  // 5. this node's id, its record, and the jobs of its inner children
  if (tid == 0) {
    const uint32_t split = b + n_left;               // split position in [1, n-1]
    uint32_t id;
    if (job.parent_slot == 0xFFFFFFFFu) {
      id = 0;
      *root_split = split;
    } else {
      const uint32_t rs = *root_split;                // written one level earlier
      id = split == 1 ? rs - 1 : split - 1;
      // hand the id to the parent's child slot
      const uint32_t p = job.parent_slot >> 1, slot = job.parent_slot & 1u;
      reinterpret_cast<int32_t*>(out + 4 * (size_t)p + 3)[slot] = (int32_t)id;
    }
    if (id >= n - 1) { atomicOr(err, ERR_BUILD); return; }
    float4* o = out + 4 * (size_t)id;
    o[0] = make_float4(cl[0][0], ch[0][0], cl[0][1], ch[0][1]);
    o[1] = make_float4(cl[1][0], ch[1][0], cl[1][1], ch[1][1]);
    o[2] = make_float4(cl[0][2], ch[0][2], cl[1][2], ch[1][2]);
    int32_t child[2] = {0, 0};
    const uint32_t rb[2] = {b, split}, re[2] = {split, e};
    for (int c = 0; c < 2; ++c) {
      if (re[c] - rb[c] == 1) {
        child[c] = ~(int32_t)idx_out[rb[c]];
      } else {
        const uint32_t at = atomicAdd(next_count, 1u);
        if (at >= n / 2 + 1) { atomicOr(err, ERR_BUILD); continue; }
        next[at] = Job{rb[c], re[c], id << 1 | (uint32_t)c, job.depth + 1};
        child[c] = 0;                                 // filled in by the child
      }
    }
    o[3] = make_float4(__int_as_float(child[0]), __int_as_float(child[1]), 0.f, 0.f);
  }
}

}  // namespace

size_t sah_tmp_bytes(uint32_t n) {
  const size_t nn = n ? n : 1;
  return 2 * nn * sizeof(float4) + 2 * nn * sizeof(uint32_t) + 2 * (nn / 2 + 1) * sizeof(Job) + 256;
}

cudaError_t build_sah_tree(const float4* lbvh_nodes, const int32_t* parent, uint32_t n,
                           float4* out, void* tmp, uint32_t* err, cudaStream_t st) {
  if (n < 2) return cudaMemcpyAsync(out, lbvh_nodes, 4 * sizeof(float4), cudaMemcpyDeviceToDevice, st);
  char* p = static_cast<char*>(tmp);
  float4* lo = reinterpret_cast<float4*>(p); p += (size_t)n * sizeof(float4);
  float4* hi = reinterpret_cast<float4*>(p); p += (size_t)n * sizeof(float4);
  uint32_t* idx[2];
  idx[0] = reinterpret_cast<uint32_t*>(p); p += (size_t)n * sizeof(uint32_t);
  idx[1] = reinterpret_cast<uint32_t*>(p); p += (size_t)n * sizeof(uint32_t);
  const size_t max_jobs = n / 2 + 1;
  Job* jobs[2];
  jobs[0] = reinterpret_cast<Job*>(p); p += max_jobs * sizeof(Job);
  jobs[1] = reinterpret_cast<Job*>(p); p += max_jobs * sizeof(Job);
  uint32_t* counters = reinterpret_cast<uint32_t*>(p);   // [0] next count, [1] root split
  const int g = (int)((n + 255) / 256);
  k_leaf_boxes<<<g, 256, 0, st>>>(lbvh_nodes, parent, n, lo, hi);
  k_iota<<<g, 256, 0, st>>>(idx[0], n);
  const Job root{0, n, 0xFFFFFFFFu, 0};
  cudaError_t e = cudaMemcpyAsync(jobs[0], &root, sizeof root, cudaMemcpyHostToDevice, st);
  uint32_t count = 1;
  for (int level = 0; level < kMaxDepth + 2 && count > 0 && e == cudaSuccess; ++level) {
    const int cur = level & 1;
    e = cudaMemsetAsync(counters, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) break;
    k_sah_level<<<count, kSahThreads, 0, st>>>(lo, hi, idx[cur], idx[cur ^ 1], jobs[cur], count,
                                               jobs[cur ^ 1], counters, out, counters + 1, n, err);
    e = cudaMemcpyAsync(&count, counters, sizeof count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (count > max_jobs) { count = 0; e = cudaErrorUnknown; }
  }
  if (e == cudaSuccess && count != 0) e = cudaErrorUnknown;   // deeper than the depth budget
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace rt
