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
// Scene creation with this build (GB300; upload, LBVH, SAH tree): the blob
// scene's 257k primitives 4.0 ms, the 10M-triangle terrain 77 ms (with the
// 4-wide tree built too: 4.5 ms and 95 ms; with one block per node on every
// level: 6.3 ms and 0.18 s; with 256 threads for every level and no bin
// combining: 12.2 ms and 0.49 s).
// One level of the tree per launch, one block per node of the level (nodes
// of at most kSmallLeaves leaves: their whole subtree in one warp):
//   1. centroid bounds of the node's leaves (block reduction);
//   2. kBins bins per axis: leaf count and the union of the leaf boxes
//      (shared-memory atomics on order-preserving integer images of floats,
//      one set of bins per warp, merged; the lanes of a warp that fall in one
//      bin combine their values first, as neighbouring leaves in Morton order
//      usually do);
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

#include <algorithm>

#include "rt_internal.cuh"

namespace rt {
namespace {

#ifndef RT_SAH_THREADS
#define RT_SAH_THREADS 256
#endif
#ifndef RT_SAH_THREADS_TOP
#define RT_SAH_THREADS_TOP 1024
#endif
// threads per node (block): 256 for the many nodes of the lower levels, 1024 for the levels of
// fewer than kTopJobs nodes, whose blocks each cover many leaves
constexpr int kSahThreads = RT_SAH_THREADS;
// levels with fewer nodes than kTopJobs run kSahThreadsTop threads per node:
// their few blocks cover many leaves each
constexpr int kSahThreadsTop = RT_SAH_THREADS_TOP;
constexpr uint32_t kTopJobs = 1024;
constexpr int kBins = 16;
constexpr int kMaxDepth = 60;        // median splits keep every leaf at or above this depth
constexpr int kSmallLeaves = 32;     // subtrees of at most this many leaves: one warp each (k_sah_small)

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

// SAH cost of splitting after bin s on axis a, from merged bins (counts and
// order-preserving box images); INFINITY when a side is empty
__device__ __forceinline__ float split_cost(const int (*cnt)[kBins], const int (*box)[kBins][6],
                                            float cext_a, int a, int s) {
  float llo[3] = {INFINITY, INFINITY, INFINITY}, lhi[3] = {-INFINITY, -INFINITY, -INFINITY};
  float rlo[3] = {INFINITY, INFINITY, INFINITY}, rhi[3] = {-INFINITY, -INFINITY, -INFINITY};
  int nl = 0, nr = 0;
  for (int q = 0; q < kBins; ++q) {
    const int c = cnt[a][q];
    if (!c) continue;
    float* blo = q <= s ? llo : rlo;
    float* bhi = q <= s ? lhi : rhi;
    for (int x = 0; x < 3; ++x) {
      blo[x] = fminf(blo[x], o2f(box[a][q][x]));
      bhi[x] = fmaxf(bhi[x], o2f(box[a][q][3 + x]));
    }
    if (q <= s) nl += c; else nr += c;
  }
  return (cext_a > 0.f && nl > 0 && nr > 0)
             ? half_area(llo, lhi) * (float)nl + half_area(rlo, rhi) * (float)nr
             : INFINITY;
}

// the first of equal least costs (deterministic): axis (-1 = none) and bin
__device__ __forceinline__ void pick_split(const float* cost, int* choice) {
  int best = -1;
  float bc = INFINITY;
  for (int i = 0; i < 3 * (kBins - 1); ++i)
    if (cost[i] < bc) { bc = cost[i]; best = i; }
  choice[0] = best < 0 ? -1 : best / (kBins - 1);
  choice[1] = best < 0 ? 0 : best % (kBins - 1);
}

// Step 5 of a node (one thread): its id from its split position, its record
// (child boxes cl/ch, leaf children as ~slot) and the jobs of its inner
// children, next level or small list.
__device__ void write_node(const Job& job, uint32_t n_left, const float cl[2][3], const float ch[2][3],
                          const uint32_t* __restrict__ idx_out, Job* __restrict__ next,
                          uint32_t* __restrict__ next_count, Job* __restrict__ small,
                          uint32_t* __restrict__ small_count, uint32_t out_buf, float4* __restrict__ out,
                          uint32_t* __restrict__ root_split, uint32_t n, uint32_t* __restrict__ err) {
  const uint32_t b = job.begin, e = job.end;
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
      const bool is_small = re[c] - rb[c] <= (uint32_t)kSmallLeaves;
      const uint32_t at = atomicAdd(is_small ? small_count : next_count, 1u);
      if (at >= n / 2 + 1) { atomicOr(err, ERR_BUILD); continue; }
      // a small subtree is built later by one warp from the leaf slots this
      // level wrote (idx buffer out_buf, kept in the depth field's top bit)
      (is_small ? small : next)[at] =
          Job{rb[c], re[c], id << 1 | (uint32_t)c, (job.depth + 1) | (is_small ? out_buf << 31 : 0u)};
      child[c] = 0;                                 // filled in by the child
    }
  }
  o[3] = make_float4(__int_as_float(child[0]), __int_as_float(child[1]), 0.f, 0.f);
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

template <int kSahThreads>
__global__ void __launch_bounds__(kSahThreads)
k_sah_level(const float4* __restrict__ leaf_lo, const float4* __restrict__ leaf_hi,
            const uint32_t* __restrict__ idx_in, uint32_t* __restrict__ idx_out,
            const Job* __restrict__ jobs, uint32_t n_jobs, Job* __restrict__ next,
            uint32_t* __restrict__ next_count, Job* __restrict__ small, uint32_t* __restrict__ small_count,
            uint32_t out_buf, float4* __restrict__ out, uint32_t* __restrict__ root_split,
            uint32_t n, uint32_t* __restrict__ err) {
  constexpr int kSahWarps = kSahThreads / 32;
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
      // neighbouring leaves (Morton order) mostly share a bin: the lanes of a
      // bin combine their values first and one of them updates the bin
      const uint32_t active = __activemask();
      for (int a = 0; a < 3; ++a) {
        if (!(cext[a] > 0.f)) continue;          // uniform over the block
        const int bin = min(kBins - 1, (int)((c[a] - cmin[a]) * ((float)kBins / cext[a])));
        const uint32_t grp = __match_any_sync(active, bin);
        int v[6];
        for (int q = 0; q < 3; ++q) {
          v[q] = __reduce_min_sync(grp, f2o(l3[q]));
          v[3 + q] = __reduce_max_sync(grp, f2o(h3[q]));
        }
        if ((uint32_t)(__ffs(grp) - 1) == (tid & 31)) {
          const int w = tid >> 5;
          atomicAdd(&s_cnt[w][a][bin], __popc(grp));
          for (int q = 0; q < 3; ++q) {
            atomicMin(&s_box[w][a][bin][q], v[q]);
            atomicMax(&s_box[w][a][bin][3 + q], v[3 + q]);
          }
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
      s_cost[tid] = split_cost(s_cnt[0], s_box[0], cext[a], a, s);
    }
    __syncthreads();
    if (tid == 0) pick_split(s_cost, s_choice);
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
  if (tid == 0)
    write_node(job, n_left, cl, ch, idx_out, next, next_count, small, small_count, out_buf, out,
               root_split, n, err);
}

// ---------------------------------------------------------------------------
// The top levels, where a level has few nodes of many leaves each: one block
// per node would leave most SMs idle (level 0 of a 257k-leaf scene is one
// block over every leaf), so each node's leaves are cut into S slices and the
// steps above run as five launches over (node, slice) blocks, with the
// per-node results (centroid bounds, bins, the split, left counts per slice,
// child boxes) combined in global memory by integer atomics and sums. Every
// combined value equals the one-block value (min / max / sums of integers),
// the split is chosen by the same code from the same bins, and the partition
// is stable (slices in order, each slice's lefts and rights in order), so
// the tree is the same as the one-block build's.
constexpr int kWideThreads = 512;
constexpr uint32_t kWideJobs = 32;       // levels of at most this many nodes may be sliced
constexpr uint32_t kWideMinLeaves = 16384;   // ... when their nodes average at least this many leaves
constexpr uint32_t kWideMinSlice = 1024;     // leaves per slice, at least
constexpr uint32_t kWideMaxSlices = 1024;    // (node, slice) blocks of a level, at most

struct WideNode {                        // per node of a sliced level
  int bounds[6];                         // centroid bounds (order-preserving images)
  int cnt[3][kBins];
  int box[3][kBins][6];
  int child[2][6];                       // child boxes (order-preserving images)
  int choice[2];                         // axis (-1: median), bin
  uint32_t n_left;                       // final left size
};

__device__ __forceinline__ void slice_range(const Job& job, uint32_t s, uint32_t S, uint32_t& sb,
                                            uint32_t& se) {
  const uint64_t m = job.end - job.begin;
  sb = job.begin + (uint32_t)(m * s / S);
  se = job.begin + (uint32_t)(m * (s + 1) / S);
}

__global__ void k_wide_init(WideNode* __restrict__ w, uint32_t count) {
  const uint32_t j = blockIdx.x;
  if (j >= count) return;
  WideNode& v = w[j];
  for (int i = threadIdx.x; i < 3 * kBins * 7; i += blockDim.x) {
    const int a = i / (kBins * 7), q = (i / 7) % kBins, f = i % 7;
    if (f == 6) v.cnt[a][q] = 0;
    else v.box[a][q][f] = f < 3 ? f2o(INFINITY) : f2o(-INFINITY);
  }
  if (threadIdx.x < 6) v.bounds[threadIdx.x] = threadIdx.x < 3 ? f2o(INFINITY) : f2o(-INFINITY);
  if (threadIdx.x < 12) v.child[threadIdx.x / 6][threadIdx.x % 6] =
      (threadIdx.x % 6) < 3 ? f2o(INFINITY) : f2o(-INFINITY);
}

// 1. centroid bounds
__global__ void __launch_bounds__(kWideThreads)
k_wide_bounds(const float4* __restrict__ leaf_lo, const float4* __restrict__ leaf_hi,
              const uint32_t* __restrict__ idx_in, const Job* __restrict__ jobs, uint32_t S,
              WideNode* __restrict__ w) {
  __shared__ int s_red[6];
  const uint32_t j = blockIdx.x / S, sl = blockIdx.x % S, tid = threadIdx.x;
  const Job job = jobs[j];
  uint32_t sb, se;
  slice_range(job, sl, S, sb, se);
  if (tid < 6) s_red[tid] = tid < 3 ? f2o(INFINITY) : f2o(-INFINITY);
  __syncthreads();
  float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (uint32_t i = sb + tid; i < se; i += kWideThreads) {
    const uint32_t k = idx_in[i];
    const float4 lo = leaf_lo[k], hi = leaf_hi[k];
    const float c[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
    for (int a = 0; a < 3; ++a) { clo[a] = fminf(clo[a], c[a]); chi[a] = fmaxf(chi[a], c[a]); }
  }
  for (int a = 0; a < 3; ++a) { atomicMin(&s_red[a], f2o(clo[a])); atomicMax(&s_red[3 + a], f2o(chi[a])); }
  __syncthreads();
  if (tid < 3) atomicMin(&w[j].bounds[tid], s_red[tid]);
  else if (tid < 6) atomicMax(&w[j].bounds[tid], s_red[tid]);
}

// the node's centroid frame and whether it splits at the object median
__device__ __forceinline__ bool wide_frame(const WideNode& v, const Job& job, float cmin[3], float cext[3]) {
  bool spread = false;
  for (int a = 0; a < 3; ++a) {
    cmin[a] = o2f(v.bounds[a]);
    cext[a] = o2f(v.bounds[3 + a]) - cmin[a];
    spread |= cext[a] > 0.f;
  }
  const uint32_t m = job.end - job.begin;
  const uint32_t lg = 32 - __clz(m - 1);
  return !spread || job.depth + lg >= (uint32_t)kMaxDepth - 4;
}

// 2. bins (per-warp bins of the block, merged, added to the node's)
__global__ void __launch_bounds__(kWideThreads)
k_wide_bins(const float4* __restrict__ leaf_lo, const float4* __restrict__ leaf_hi,
            const uint32_t* __restrict__ idx_in, const Job* __restrict__ jobs, uint32_t S,
            WideNode* __restrict__ w) {
  constexpr int kWarps = kWideThreads / 32;
  __shared__ int s_cnt[kWarps][3][kBins];
  __shared__ int s_box[kWarps][3][kBins][6];
  const uint32_t j = blockIdx.x / S, sl = blockIdx.x % S, tid = threadIdx.x;
  const Job job = jobs[j];
  float cmin[3], cext[3];
  if (wide_frame(w[j], job, cmin, cext)) return;         // uniform over the block
  uint32_t sb, se;
  slice_range(job, sl, S, sb, se);
  for (int i = tid; i < kWarps * 3 * kBins; i += kWideThreads) {
    const int wi = i / (3 * kBins), a = (i / kBins) % 3, q = i % kBins;
    s_cnt[wi][a][q] = 0;
    for (int c = 0; c < 6; ++c) s_box[wi][a][q][c] = c < 3 ? f2o(INFINITY) : f2o(-INFINITY);
  }
  __syncthreads();
  for (uint32_t i = sb + tid; i < se; i += kWideThreads) {
    const uint32_t k = idx_in[i];
    const float4 lo = leaf_lo[k], hi = leaf_hi[k];
    const float c[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
    const float l3[3] = {lo.x, lo.y, lo.z}, h3[3] = {hi.x, hi.y, hi.z};
    const uint32_t active = __activemask();
    for (int a = 0; a < 3; ++a) {
      if (!(cext[a] > 0.f)) continue;
      const int bin = min(kBins - 1, (int)((c[a] - cmin[a]) * ((float)kBins / cext[a])));
      const uint32_t grp = __match_any_sync(active, bin);
      int v[6];
      for (int q = 0; q < 3; ++q) {
        v[q] = __reduce_min_sync(grp, f2o(l3[q]));
        v[3 + q] = __reduce_max_sync(grp, f2o(h3[q]));
      }
      if ((uint32_t)(__ffs(grp) - 1) == (tid & 31)) {
        const int wi = tid >> 5;
        atomicAdd(&s_cnt[wi][a][bin], __popc(grp));
        for (int q = 0; q < 3; ++q) {
          atomicMin(&s_box[wi][a][bin][q], v[q]);
          atomicMax(&s_box[wi][a][bin][3 + q], v[3 + q]);
        }
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < 3 * kBins * 7; i += kWideThreads) {
    const int a = i / (kBins * 7), q = (i / 7) % kBins, f = i % 7;
    if (f == 6) {
      int t = 0;
      for (int wi = 0; wi < kWarps; ++wi) t += s_cnt[wi][a][q];
      if (t) atomicAdd(&w[j].cnt[a][q], t);
    } else {
      int v = s_box[0][a][q][f];
      for (int wi = 1; wi < kWarps; ++wi) v = f < 3 ? min(v, s_box[wi][a][q][f]) : max(v, s_box[wi][a][q][f]);
      if (f < 3) { if (v != f2o(INFINITY)) atomicMin(&w[j].box[a][q][f], v); }
      else if (v != f2o(-INFINITY)) atomicMax(&w[j].box[a][q][f], v);
    }
  }
}

// the node's split from its merged bins (every block of the node the same)
__device__ void wide_choice(const WideNode& v, const Job& job, float cmin[3], float cext[3],
                            float* s_cost, int* s_choice) {
  const uint32_t tid = threadIdx.x;
  const bool median = wide_frame(v, job, cmin, cext);
  if (!median && tid < 3 * (kBins - 1)) {
    const int a = tid / (kBins - 1), s = tid % (kBins - 1);
    s_cost[tid] = split_cost(v.cnt, v.box, cext[a], a, s);
  }
  __syncthreads();
  if (tid == 0) {
    if (median) { s_choice[0] = -1; s_choice[1] = 0; }
    else pick_split(s_cost, s_choice);
  }
  __syncthreads();
}

__device__ __forceinline__ bool goes_left(const float4& lo, const float4& hi, int axis, int split_bin,
                                          const float cmin[3], const float cext[3]) {
  const float c = 0.5f * ((&lo.x)[axis] + (&hi.x)[axis]);
  return min(kBins - 1, (int)((c - cmin[axis]) * ((float)kBins / cext[axis]))) <= split_bin;
}

// 3. the split, and the left count of each slice
__global__ void __launch_bounds__(kWideThreads)
k_wide_count(const float4* __restrict__ leaf_lo, const float4* __restrict__ leaf_hi,
             const uint32_t* __restrict__ idx_in, const Job* __restrict__ jobs, uint32_t S,
             WideNode* __restrict__ w, uint32_t* __restrict__ slice_left) {
  __shared__ float s_cost[3 * (kBins - 1)];
  __shared__ int s_choice[2];
  __shared__ uint32_t s_sum;
  const uint32_t j = blockIdx.x / S, sl = blockIdx.x % S, tid = threadIdx.x;
  const Job job = jobs[j];
  float cmin[3], cext[3];
  wide_choice(w[j], job, cmin, cext, s_cost, s_choice);
  const int axis = s_choice[0], split_bin = s_choice[1];
  if (sl == 0 && tid == 0) { w[j].choice[0] = axis; w[j].choice[1] = split_bin; }
  if (axis < 0) return;
  uint32_t sb, se;
  slice_range(job, sl, S, sb, se);
  if (tid == 0) s_sum = 0;
  __syncthreads();
  uint32_t c = 0;
  for (uint32_t i = sb + tid; i < se; i += kWideThreads) {
    const uint32_t k = idx_in[i];
    c += goes_left(leaf_lo[k], leaf_hi[k], axis, split_bin, cmin, cext) ? 1u : 0u;
  }
  c = __reduce_add_sync(0xFFFFFFFFu, c);
  if ((tid & 31) == 0) atomicAdd(&s_sum, c);
  __syncthreads();
  if (tid == 0) slice_left[blockIdx.x] = s_sum;
}

// 4. stable scatter of each slice (lefts, then rights, in order) and the
//    child boxes
__global__ void __launch_bounds__(kWideThreads)
k_wide_scatter(const float4* __restrict__ leaf_lo, const float4* __restrict__ leaf_hi,
               const uint32_t* __restrict__ idx_in, uint32_t* __restrict__ idx_out,
               const Job* __restrict__ jobs, uint32_t S, WideNode* __restrict__ w,
               const uint32_t* __restrict__ slice_left) {
  constexpr int kWarps = kWideThreads / 32;
  __shared__ uint32_t s_scan[kWarps];
  __shared__ int s_red[12];
  const uint32_t j = blockIdx.x / S, sl = blockIdx.x % S, tid = threadIdx.x;
  const uint32_t lane = tid & 31, warp = tid >> 5;
  const Job job = jobs[j];
  const uint32_t b = job.begin, m = job.end - job.begin;
  float cmin[3], cext[3];
  wide_frame(w[j], job, cmin, cext);
  const int axis = w[j].choice[0], split_bin = w[j].choice[1];
  uint32_t before = 0, n_left = 0;
  if (axis >= 0)
    for (uint32_t q = 0; q < S; ++q) {
      const uint32_t v = slice_left[j * S + q];
      if (q < sl) before += v;
      n_left += v;
    }
  // an empty side cannot happen (the scatter repeats the binning
  // arithmetic); the object median stands in, as in the one-block build
  const bool median = axis < 0 || n_left == 0 || n_left == m;
  if (median) n_left = m / 2;
  if (sl == 0 && tid == 0) w[j].n_left = n_left;
  uint32_t sb, se;
  slice_range(job, sl, S, sb, se);
  if (tid < 12) s_red[tid] = (tid % 6) < 3 ? f2o(INFINITY) : f2o(-INFINITY);
  float l[2][3], h[2][3];
  for (int c = 0; c < 2; ++c)
    for (int x = 0; x < 3; ++x) { l[c][x] = INFINITY; h[c][x] = -INFINITY; }
  uint32_t cnt_left = 0;
  const uint32_t rights_before = (sb - b) - before;
  for (uint32_t base = sb; base < se; base += kWideThreads) {
    const uint32_t i = base + tid;
    bool left = false;
    uint32_t k = 0;
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
    if (i < se) {
      k = idx_in[i];
      lo = leaf_lo[k];
      hi = leaf_hi[k];
      left = median ? (i - b) < n_left : goes_left(lo, hi, axis, split_bin, cmin, cext);
    }
    const uint32_t ball = __ballot_sync(0xFFFFFFFFu, left);
    __syncthreads();
    if (lane == 0) s_scan[warp] = __popc(ball);
    __syncthreads();
    uint32_t wb = 0, chunk = 0;
    for (uint32_t q = 0; q < (uint32_t)kWarps; ++q) {
      if (q < warp) wb += s_scan[q];
      chunk += s_scan[q];
    }
    const uint32_t rank = wb + __popc(ball & ((1u << lane) - 1u));   // lefts before i in the chunk
    if (i < se) {
      const uint32_t t = i - base;
      if (median) idx_out[i] = k;
      else if (left) idx_out[b + before + cnt_left + rank] = k;
      else idx_out[b + n_left + rights_before + ((base - sb) - cnt_left) + (t - rank)] = k;
      const int c = left ? 0 : 1;
      l[c][0] = fminf(l[c][0], lo.x); l[c][1] = fminf(l[c][1], lo.y); l[c][2] = fminf(l[c][2], lo.z);
      h[c][0] = fmaxf(h[c][0], hi.x); h[c][1] = fmaxf(h[c][1], hi.y); h[c][2] = fmaxf(h[c][2], hi.z);
    }
    cnt_left += chunk;
  }
  for (int c = 0; c < 2; ++c)
    for (int x = 0; x < 3; ++x) {
      atomicMin(&s_red[6 * c + x], f2o(l[c][x]));
      atomicMax(&s_red[6 * c + 3 + x], f2o(h[c][x]));
    }
  __syncthreads();
  if (tid < 12) {
    const int c = tid / 6, f = tid % 6;
    if (f < 3) { if (s_red[tid] != f2o(INFINITY)) atomicMin(&w[j].child[c][f], s_red[tid]); }
    else if (s_red[tid] != f2o(-INFINITY)) atomicMax(&w[j].child[c][f], s_red[tid]);
  }
}

// 5. the node records and the next jobs (one thread per node)
__global__ void k_wide_nodes(const Job* __restrict__ jobs, uint32_t count, const WideNode* __restrict__ w,
                             const uint32_t* __restrict__ idx_out, Job* __restrict__ next,
                             uint32_t* __restrict__ next_count, Job* __restrict__ small,
                             uint32_t* __restrict__ small_count, uint32_t out_buf, float4* __restrict__ out,
                             uint32_t* __restrict__ root_split, uint32_t n, uint32_t* __restrict__ err) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= count) return;
  float cl[2][3], ch[2][3];
  for (int c = 0; c < 2; ++c)
    for (int x = 0; x < 3; ++x) { cl[c][x] = o2f(w[j].child[c][x]); ch[c][x] = o2f(w[j].child[c][3 + x]); }
  write_node(jobs[j], w[j].n_left, cl, ch, idx_out, next, next_count, small, small_count, out_buf, out,
             root_split, n, err);
}

// warp-wide inclusive scan of a box (lanes in order), forward or backward
__device__ __forceinline__ void box_scan(float lo[3], float hi[3], bool backward) {
  const uint32_t lane = threadIdx.x & 31;
  for (int o = 1; o < 32; o <<= 1) {
    float l[3], h[3];
    for (int x = 0; x < 3; ++x) {
      l[x] = backward ? __shfl_down_sync(0xFFFFFFFFu, lo[x], o) : __shfl_up_sync(0xFFFFFFFFu, lo[x], o);
      h[x] = backward ? __shfl_down_sync(0xFFFFFFFFu, hi[x], o) : __shfl_up_sync(0xFFFFFFFFu, hi[x], o);
    }
    const bool ok = backward ? lane + o < 32 : lane >= (uint32_t)o;
    if (ok)
      for (int x = 0; x < 3; ++x) { lo[x] = fminf(lo[x], l[x]); hi[x] = fmaxf(hi[x], h[x]); }
  }
}

// Subtrees of at most kSmallLeaves leaves, one warp each: every node takes
// the split of least SAH cost over all positions of its leaves sorted by
// centroid on each axis (a warp bitonic sort, ties by leaf order, then box
// prefix and suffix scans), or the median of the current order when the
// depth budget is short. Node ids follow the split positions as in
// k_sah_level.
constexpr int kSmallWarps = 4;
__global__ void __launch_bounds__(32 * kSmallWarps)
k_sah_small(const float4* __restrict__ leaf_lo, const float4* __restrict__ leaf_hi,
            uint32_t* const* __restrict__ idx_bufs, const Job* __restrict__ jobs, uint32_t n_jobs,
            float4* __restrict__ out, const uint32_t* __restrict__ root_split, uint32_t n,
            uint32_t* __restrict__ err) {
  __shared__ uint32_t s_slot[kSmallWarps][kSmallLeaves];     // leaf slots in the current order
  __shared__ float s_box[kSmallWarps][kSmallLeaves][6];
  __shared__ uint32_t s_tmp[kSmallWarps][kSmallLeaves];
  __shared__ float s_tbox[kSmallWarps][kSmallLeaves][6];
  __shared__ Job s_stack[kSmallWarps][kSmallLeaves];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t j = blockIdx.x * kSmallWarps + warp;
  if (j >= n_jobs) return;
  const Job job = jobs[j];
  const uint32_t base = job.begin, m = job.end - job.begin;
  const uint32_t* idx = idx_bufs[job.depth >> 31];
  if (m < 2 || m > (uint32_t)kSmallLeaves) { if (lane == 0) atomicOr(err, ERR_BUILD); return; }
  const uint32_t rs = *root_split;
  if (lane < m) {
    const uint32_t k = idx[base + lane];
    s_slot[warp][lane] = k;
    const float4 lo = leaf_lo[k], hi = leaf_hi[k];
    s_box[warp][lane][0] = lo.x; s_box[warp][lane][1] = lo.y; s_box[warp][lane][2] = lo.z;
    s_box[warp][lane][3] = hi.x; s_box[warp][lane][4] = hi.y; s_box[warp][lane][5] = hi.z;
  }
  int sp = 0;
  if (lane == 0) s_stack[warp][0] = Job{0, m, job.parent_slot, job.depth & 0x7FFFFFFFu};
  sp = 1;
  __syncwarp();
  for (uint32_t guard = 0; sp > 0 && guard < 2 * kSmallLeaves; ++guard) {
    const Job t = s_stack[warp][--sp];
    __syncwarp();
    const uint32_t b = t.begin, s = t.end - t.begin;
    const bool in = lane < s;
    float blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (in)
      for (int x = 0; x < 3; ++x) { blo[x] = s_box[warp][b + lane][x]; bhi[x] = s_box[warp][b + lane][3 + x]; }
    uint32_t k_split = s / 2;                 // median of the current order unless the SAH wins
    int best_axis = -1;
    float best_cost = INFINITY;
    if (t.depth + s - 1 <= (uint32_t)kMaxDepth) {
      for (int axis = 0; axis < 3; ++axis) {
        // sort (centroid, position) ascending over the lanes; out-of-range lanes last
        float key = in ? 0.5f * (blo[axis] + bhi[axis]) : INFINITY;
        uint32_t val = in ? lane : 0xFFFFFFFFu;
        for (uint32_t kk = 2; kk <= 32; kk <<= 1)
          for (uint32_t jj = kk >> 1; jj > 0; jj >>= 1) {
            const float ok = __shfl_xor_sync(0xFFFFFFFFu, key, jj);
            const uint32_t ov = __shfl_xor_sync(0xFFFFFFFFu, val, jj);
            const bool up = (lane & kk) == 0, lower = (lane & jj) == 0;
            const bool other_less = ok < key || (ok == key && ov < val);
            const bool take = (lower == up) ? other_less : !other_less && !(ok == key && ov == val);
            if (take) { key = ok; val = ov; }
          }
        // boxes in sorted order; prefix and suffix unions
        float plo[3], phi[3], qlo[3], qhi[3];
        for (int x = 0; x < 3; ++x) {
          const float vlo = val < s ? s_box[warp][b + val][x] : INFINITY;
          const float vhi = val < s ? s_box[warp][b + val][3 + x] : -INFINITY;
          plo[x] = qlo[x] = vlo; phi[x] = qhi[x] = vhi;
        }
        box_scan(plo, phi, false);
        box_scan(qlo, qhi, true);
        // split after sorted position lane (left lane+1 leaves)
        float q2lo[3], q2hi[3];
        for (int x = 0; x < 3; ++x) {
          q2lo[x] = __shfl_down_sync(0xFFFFFFFFu, qlo[x], 1);
          q2hi[x] = __shfl_down_sync(0xFFFFFFFFu, qhi[x], 1);
        }
        float cost = INFINITY;
        if (lane + 1 < s)
          cost = half_area(plo, phi) * (float)(lane + 1) + half_area(q2lo, q2hi) * (float)(s - lane - 1);
        // warp argmin, lowest position among equal costs
        float bc = cost;
        uint32_t bl = lane;
        for (int o = 16; o > 0; o >>= 1) {
          const float c2 = __shfl_xor_sync(0xFFFFFFFFu, bc, o);
          const uint32_t l2 = __shfl_xor_sync(0xFFFFFFFFu, bl, o);
          if (c2 < bc || (c2 == bc && l2 < bl)) { bc = c2; bl = l2; }
        }
        if (bc < best_cost) {               // warp-uniform
          best_cost = bc;
          best_axis = axis;
          k_split = bl + 1;
          // keep this axis's order
          if (in) {
            s_tmp[warp][lane] = s_slot[warp][b + val];
            for (int x = 0; x < 6; ++x) s_tbox[warp][lane][x] = s_box[warp][b + val][x];
          }
        }
        __syncwarp();
      }
      if (best_axis >= 0 && in) {
        s_slot[warp][b + lane] = s_tmp[warp][lane];
        for (int x = 0; x < 6; ++x) s_box[warp][b + lane][x] = s_tbox[warp][lane][x];
      }
      __syncwarp();
    }
    // child boxes of the split at k_split in the current order
    float c0lo[3], c0hi[3], c1lo[3], c1hi[3];
    for (int x = 0; x < 3; ++x) {
      const bool l0 = in && lane < k_split, l1 = in && lane >= k_split;
      const float vlo = in ? s_box[warp][b + lane][x] : INFINITY, vhi = in ? s_box[warp][b + lane][3 + x] : -INFINITY;
      float a0 = l0 ? vlo : INFINITY, a1 = l1 ? vlo : INFINITY, z0 = l0 ? vhi : -INFINITY, z1 = l1 ? vhi : -INFINITY;
      for (int o = 16; o > 0; o >>= 1) {
        a0 = fminf(a0, __shfl_xor_sync(0xFFFFFFFFu, a0, o));
        a1 = fminf(a1, __shfl_xor_sync(0xFFFFFFFFu, a1, o));
        z0 = fmaxf(z0, __shfl_xor_sync(0xFFFFFFFFu, z0, o));
        z1 = fmaxf(z1, __shfl_xor_sync(0xFFFFFFFFu, z1, o));
      }
      c0lo[x] = a0; c1lo[x] = a1; c0hi[x] = z0; c1hi[x] = z1;
    }
    if (lane == 0) {
      const uint32_t split = base + b + k_split;      // global split position
      const uint32_t id = split == 1 ? rs - 1 : split - 1;
      reinterpret_cast<int32_t*>(out + 4 * (size_t)(t.parent_slot >> 1) + 3)[t.parent_slot & 1u] = (int32_t)id;
      if (id < n - 1) {
        float4* o = out + 4 * (size_t)id;
        o[0] = make_float4(c0lo[0], c0hi[0], c0lo[1], c0hi[1]);
        o[1] = make_float4(c1lo[0], c1hi[0], c1lo[1], c1hi[1]);
        o[2] = make_float4(c0lo[2], c0hi[2], c1lo[2], c1hi[2]);
        const uint32_t rb[2] = {b, b + k_split}, re[2] = {b + k_split, b + s};
        int32_t child[2];
        for (int c = 0; c < 2; ++c) {
          if (re[c] - rb[c] == 1) {
            child[c] = ~(int32_t)s_slot[warp][rb[c]];
          } else {
            child[c] = 0;                       // filled in when the child is built
            s_stack[warp][sp + c] = Job{rb[c], re[c], id << 1 | (uint32_t)c, t.depth + 1};
          }
        }
        o[3] = make_float4(__int_as_float(child[0]), __int_as_float(child[1]), 0.f, 0.f);
      } else {
        atomicOr(err, ERR_BUILD);
      }
    }
    __syncwarp();
    // the pushes lane 0 made (warp-uniform count)
    sp += (k_split > 1 ? 1 : 0) + (s - k_split > 1 ? 1 : 0);
    if (k_split == 1 && s - k_split > 1) {      // only the right child was pushed, at sp + 1
      if (lane == 0) s_stack[warp][sp - 1] = s_stack[warp][sp];
    }
    __syncwarp();
  }
  if (sp != 0 && lane == 0) atomicOr(err, ERR_BUILD);
}

}  // namespace

namespace {
bool g_sah_slicing = true;
}  // namespace

void set_sah_slicing(bool on) { g_sah_slicing = on; }

size_t sah_tmp_bytes(uint32_t n) {
  const size_t nn = n ? n : 1;
  return 2 * nn * sizeof(float4) + 2 * nn * sizeof(uint32_t) + 3 * (nn / 2 + 1) * sizeof(Job) + 256 +
         kWideJobs * sizeof(WideNode) + kWideMaxSlices * sizeof(uint32_t) + 256;
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
  Job* small = reinterpret_cast<Job*>(p); p += max_jobs * sizeof(Job);
  uint32_t** d_bufs = reinterpret_cast<uint32_t**>(p); p += 2 * sizeof(uint32_t*);
  uint32_t* counters = reinterpret_cast<uint32_t*>(p);   // [0] next count, [1] root split, [2] small count
  p += 256 - 2 * sizeof(uint32_t*);
  WideNode* wide = reinterpret_cast<WideNode*>(p); p += kWideJobs * sizeof(WideNode);
  uint32_t* slice_left = reinterpret_cast<uint32_t*>(p);
  const int g = (int)((n + 255) / 256);
  k_leaf_boxes<<<g, 256, 0, st>>>(lbvh_nodes, parent, n, lo, hi);
  k_iota<<<g, 256, 0, st>>>(idx[0], n);
  const Job root{0, n, 0xFFFFFFFFu, 0};
  cudaError_t e = cudaMemcpyAsync(jobs[0], &root, sizeof root, cudaMemcpyHostToDevice, st);
  uint32_t* h_bufs[2] = {idx[0], idx[1]};
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_bufs, h_bufs, sizeof h_bufs, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(counters + 2, 0, sizeof(uint32_t), st);
  uint32_t count = 1;
  for (int level = 0; level < kMaxDepth + 2 && count > 0 && e == cudaSuccess; ++level) {
    const int cur = level & 1;
    e = cudaMemsetAsync(counters, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) break;
    // few nodes of many leaves each: slice every node over several blocks
    const uint32_t per_job = n / count;
    if (g_sah_slicing && count <= kWideJobs && per_job >= kWideMinLeaves) {
      uint32_t S = (2u * (uint32_t)num_sms() + count - 1) / count;
      S = std::min(S, std::min(per_job / kWideMinSlice, kWideMaxSlices / count));
      S = std::max(S, 1u);
      const uint32_t blocks = count * S;
      k_wide_init<<<count, 256, 0, st>>>(wide, count);
      k_wide_bounds<<<blocks, kWideThreads, 0, st>>>(lo, hi, idx[cur], jobs[cur], S, wide);
      k_wide_bins<<<blocks, kWideThreads, 0, st>>>(lo, hi, idx[cur], jobs[cur], S, wide);
      k_wide_count<<<blocks, kWideThreads, 0, st>>>(lo, hi, idx[cur], jobs[cur], S, wide, slice_left);
      k_wide_scatter<<<blocks, kWideThreads, 0, st>>>(lo, hi, idx[cur], idx[cur ^ 1], jobs[cur], S, wide,
                                                      slice_left);
      k_wide_nodes<<<(count + 31) / 32, 32, 0, st>>>(jobs[cur], count, wide, idx[cur ^ 1], jobs[cur ^ 1],
                                                     counters, small, counters + 2, (uint32_t)(cur ^ 1),
                                                     out, counters + 1, n, err);
    } else if (count < kTopJobs)
      k_sah_level<kSahThreadsTop><<<count, kSahThreadsTop, 0, st>>>(
          lo, hi, idx[cur], idx[cur ^ 1], jobs[cur], count, jobs[cur ^ 1], counters, small,
          counters + 2, (uint32_t)(cur ^ 1), out, counters + 1, n, err);
    else
      k_sah_level<kSahThreads><<<count, kSahThreads, 0, st>>>(
          lo, hi, idx[cur], idx[cur ^ 1], jobs[cur], count, jobs[cur ^ 1], counters, small,
          counters + 2, (uint32_t)(cur ^ 1), out, counters + 1, n, err);
    e = cudaMemcpyAsync(&count, counters, sizeof count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (count > max_jobs) { count = 0; e = cudaErrorUnknown; }
  }
  if (e == cudaSuccess && count != 0) e = cudaErrorUnknown;   // deeper than the depth budget
  uint32_t n_small = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&n_small, counters + 2, sizeof n_small, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && n_small > max_jobs) e = cudaErrorUnknown;
  if (e == cudaSuccess && n_small > 0)
    k_sah_small<<<(n_small + kSmallWarps - 1) / kSmallWarps, 32 * kSmallWarps, 0, st>>>(
        lo, hi, d_bufs, small, n_small, out, counters + 1, n, err);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace rt
