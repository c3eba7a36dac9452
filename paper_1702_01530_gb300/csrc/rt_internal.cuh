// Internal declarations of the GB300 stereo ray tracer (CUDA, sm_103a).
//
// Data layout in HBM (all 16-byte aligned, read with 16-byte vector loads):
//   nodes  : (n-1) BVH2 nodes of 64 B = 4 x float4, binary radix tree
//            numbering (root 0). Both children's boxes live in the parent:
//              [0] = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//              [1] = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//              [2] = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//              [3] = (left, right, -, -) as int bits; >= 0 internal, < 0 leaf ~k
//   prims  : n leaf records of 48 B = 3 x float4 in leaf (sorted key) order:
//            triangle: (v0.xyz, id) (e1.xyz, material) (e2.xyz, 0)
//            sphere  : (c.xyz, id)  (r, 0, 0, material)  (0, 0, 0, 0)
//            (id and material stored as uint bits; id < n_spheres = sphere)
//   mats   : float4 (albedo rgb, reflectivity)
//   lights : float4 (position xyz, intensity)
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/rt_stereo.h"

namespace rt {

// device error word bits
enum : uint32_t {
  ERR_STACK = 1u,      // traversal stack bound exceeded
  ERR_ITER = 2u,       // traversal iteration bound reached
  ERR_QUEUE = 4u,      // a wavefront queue would overflow
  ERR_INDEX = 8u,      // an index read from memory is out of range
  ERR_BUILD = 16u,     // BVH refit did not reach the root
};

// the tree a render walks
constexpr int kTreeBinary = 0, kTreeWide4 = 1;

constexpr int kStackSize = 64;   // >= the depth of the LBVH (64-bit keys) and of the SAH tree (60)
constexpr int32_t kEmptyChild = 0x7FFFFFFF;  // unused slot of a 4-wide node
constexpr float kAmbient = 0.1f;
constexpr float kBgR = 0.2f, kBgG = 0.3f, kBgB = 0.5f;

struct DeviceScene {
  const float4* nodes;
  const float4* nodes4;   // 4-wide nodes (7 float4 each), the top n_top first
  const float4* prims;
  const float4* mats;
  const float4* lights;
  uint32_t n_prims, n_spheres, n_mats, n_lights;
  uint32_t n4, n_top;     // 4-wide nodes, of which the first n_top are staged in shared memory
};

// host-computed camera basis (double -> float)
struct CameraParams {
  float eye[3], right[3], up[3], fwd[3];
  float tan_x, tan_y, zc, half_sep;
  float sx, sy;                // 2 tan_x / W and 2 tan_y / H (pixel step in window units)
  uint32_t W, H;              // the whole image (it fixes the rays)
  uint32_t tiles_x, tiles_y;  // 8x4-pixel tiles per eye (of the traced rows)
  uint32_t y0, rows;          // the rows traced: y0 .. y0 + rows - 1 (0 and H for a whole image)
};

// stages of one render, in launch order
enum Stage : int {
  ST_CLEAR = 0,     // counter and accumulator clears
  ST_TRACE = 1,     // all rays: primary, shadow and mirror (one persistent kernel)
  ST_RESOLVE = 2,   // fixed-point sums to float RGB
  ST_WARP = 3,      // reprojection: forward warp and features
  ST_NET = 4,       // reprojection: retrace network
  ST_MASK = 5,      // reprojection: retrace mask and compaction
  ST_RETRACE = 6,   // reprojection: tracing the masked right pixels
  ST_COMPOSE = 7,   // reprojection: right image composition
  ST_COUNT = 8
};
constexpr int kMaxEvents = 24;

// reprojection scratch of a scene (per right-eye pixel unless noted)
struct ReprojBuffers {
  void* base = nullptr;
  uint64_t cap = 0;              // pixels per eye the buffers hold
  float* depth_L = nullptr;      // left G-buffer: view depth, normal (3), hit id
  float* normal_L = nullptr;
  float* refl_L = nullptr;       // reflectivity of the left primary hit (0 on a miss)
  uint32_t* id_L = nullptr;
  unsigned long long* zbuf = nullptr;  // forward-warp z-test keys
  __nv_bfloat16* feat16 = nullptr;     // network input, 16 channels
  uint8_t* hole = nullptr;
  float* warped = nullptr;       // warped left RGB (3)
  uint8_t* mask = nullptr;       // retrace mask
  uint32_t* plist = nullptr;     // masked pixels (global indices)
  uint32_t* count = nullptr;     // number of masked pixels
  float* prob = nullptr;         // network output
  __nv_bfloat16* act[3] = {nullptr, nullptr, nullptr};  // hidden activations (32 channels)
};

// scratch of one render (scene-owned, grown on demand)
struct Workspace {
  size_t bytes = 0;
  void* base = nullptr;
  uint32_t* accum = nullptr;     // 2*P*3 fixed-point colour sums
  float4* wq = nullptr;          // warp queues: n_warps x (cap_s + cap_r) x 3 float4
  float4* pool = nullptr;        // drain pools: shadow then mirror, cap_p entries of 3 float4 each
  uint32_t* pool_flag = nullptr; // per pool entry: epoch of the render that wrote it
  uint32_t cap_p = 0;            // entries per drain pool
  uint32_t cap_p_limit = 0;      // test hook: renders use at most this many (0 = cap_p)
  uint32_t epoch = 0;            // renders issued on this workspace (pool flags hold it)
  uint32_t* counters = nullptr;  // see Counter enum
  uint32_t cap_s = 0, cap_r = 0; // shadow / mirror entries per warp
  uint64_t n_warps = 0;          // warps the queues are sized for
  uint64_t cap_pixels = 0;       // 2*P the accumulators are sized for
  float4* frame = nullptr;       // frame buffers for rt_render_stereo_host
  size_t frame_bytes = 0;
  // rt_render_stereo_sequence: two device frame slots (each both images),
  // a copy stream and per slot the events "rendered" and "copied"
  float* seq_frame = nullptr;
  size_t seq_frame_bytes = 0;    // bytes of one slot
  cudaStream_t seq_copy = nullptr;
  cudaEvent_t seq_rendered[2] = {}, seq_copied[2] = {};
  uint32_t L = 0;
  ReprojBuffers rp;
  // stage timing (CUDA events on the render stream), see Stage
  bool profile = false;
  cudaEvent_t ev[kMaxEvents] = {};
  int ev_stage[kMaxEvents] = {};  // stage that ends at event k
  int n_ev = 0;
};

// counters block layout (uint32 each)
// (one 128-byte line each: the tile counter that every warp hammers, a flag
// that changes once, and the drain-pool counters)
enum Counter : int {
  C_TILE = 0,       // next primary tile
  C_SHADOW = 1,     // shadow rays enqueued (all warps)
  C_REFL = 2,       // mirror rays enqueued (all warps)
  C_TILES_OUT = 32, // set once a warp has found every tile handed out
  C_S_AVAIL = 64,   // drain pools: published entries not yet taken (int32), shadow
  C_R_AVAIL = 65,   // ... mirror
  C_S_HEAD = 66,    // drain pools: next entry to take / next entry to reserve, shadow
  C_S_TAIL = 67,
  C_R_HEAD = 68,    // ... mirror
  C_R_TAIL = 69,
  C_TOTAL = 96
};

struct RenderArgs {
  DeviceScene sc;
  CameraParams cam;
  uint32_t max_depth;
  float color_scale;       // fixed-point scale of the colour accumulators
  float* out_L;
  float* out_R;
  uint32_t* hit_L;
  uint32_t* hit_R;
  float* depth_L;
  float* depth_R;
  float* normal_L;         // G-buffer: primary-hit normal (facing the ray), 3 floats/pixel
  float* refl_L;           // G-buffer: reflectivity of the left primary hit (0 on a miss)
  float* normal_R;
  uint64_t* ray_counts;
  uint64_t* work;          // non-null => instrumented traversal
  uint32_t* err;           // device error word
  uint32_t eyes;           // 1 = left only, 2 = right only, 3 = both
  const uint32_t* plist;   // optional list of pixels to trace (eye*P + y*W + x)
  uint32_t plist_n;        // its length, or
  const uint32_t* plist_n_dev;  // its length in device memory (read by the kernel)
  bool resolve;            // write out_L/out_R from the sums (false: caller composes)
  int trace_stage;         // stage the tracing kernel is timed as (ST_TRACE or ST_RETRACE)
  int tree;                // kTreeBinary (sc.nodes) or kTreeWide4 (sc.nodes4)
  // several frames in one launch (0 or 1: just cam): n_frames cameras of the
  // same image size in host memory (frames[0] is cam); pixel ids, sums,
  // images and G-buffers then run over all frames, eye-major:
  // eye * (n_frames P) + frame * P + pixel
  uint32_t n_frames;
  const CameraParams* frames;
};
constexpr int kMaxFrames = 8;

// entry points implemented in the .cu files
cudaError_t build_lbvh(const float4* d_sph_in, const float* d_tri_in, uint32_t ns, uint32_t nt,
                       float4* d_nodes, float4* d_prims, uint64_t* d_keys, int32_t* d_parent,
                       void* d_tmp, size_t tmp_bytes, uint32_t* d_err, cudaStream_t st);
size_t lbvh_tmp_bytes(uint32_t n);
size_t sah_tmp_bytes(uint32_t n);
// binned-SAH binary tree over the leaves of the LBVH (nodes, parent): same
// node layout and leaf slots, root 0; synchronises st once per tree level
cudaError_t build_sah_tree(const float4* lbvh_nodes, const int32_t* parent, uint32_t n,
                           float4* out, void* tmp, uint32_t* err, cudaStream_t st);
size_t bvh4_tmp_bytes(uint32_t n);
void set_sah_slicing(bool on);   // slice the top levels of the SAH build (default on)
cudaError_t inner_parents(const float4* nodes, uint32_t n, int32_t* parent, cudaStream_t st);
cudaError_t build_bvh4(const float4* nodes, const int32_t* parent, uint32_t n, int top_depth,
                       float4* nodes4, uint32_t* counts_dev, void* tmp, cudaStream_t st);
cudaError_t render(const RenderArgs& a, Workspace& ws, cudaStream_t st);
// stage timing: start a profiled call (resets the event list) / mark the end of a stage
void profile_begin(Workspace& ws, cudaStream_t st);
void profile_mark(Workspace& ws, int stage, cudaStream_t st);
int num_sms();
int render_grid();      // persistent blocks of the render kernel
int render_threads();   // threads per block of the render kernel
int treelet_depth();    // 4-wide levels numbered first for shared-memory staging

// reprojection (reproj.cu)
cudaError_t reproj_warp(const float* depth_L, const float* normal_L, const uint32_t* id_L,
                        const float* rgb_L, const float* refl_L, uint32_t W, uint32_t H, float f_px, float eye_sep,
                        float convergence, unsigned long long* zbuf, __nv_bfloat16* feat16,
                        float* feat32, uint8_t* hole, float* warped, cudaStream_t st);
cudaError_t reproj_labels(const uint8_t* hole, const float* warped, const float* full_R, uint32_t P,
                          float thr, float* label, cudaStream_t st);
cudaError_t reproj_mask(const uint8_t* hole, const float* prob, uint32_t P, float threshold,
                        uint8_t* mask, uint32_t* plist, uint32_t* count, cudaStream_t st);
cudaError_t reproj_compose(const uint8_t* mask, const uint32_t* accum_R, const float* warped,
                           uint32_t P, float inv_scale, float* out_R, cudaStream_t st);

// retrace network (nn.cu)
namespace nn {
constexpr uint32_t kParams = 21697;
void set_conv_smem_pad(int bytes);
size_t packed_fwd_elems(int l);
size_t packed_bwd_elems(int l);
cudaError_t pack_weights(const float* params, __nv_bfloat16* const wf[4], __nv_bfloat16* const wb[4],
                         cudaStream_t st);
// forward / forward_fp8: n_img feature maps of W x H pixels each, stacked
// image after image (one launch per layer for all of them)
cudaError_t forward(const __nv_bfloat16* feat16, const float* params, __nv_bfloat16* const wf[4],
                    __nv_bfloat16* act1, __nv_bfloat16* act2, __nv_bfloat16* act3, float* prob,
                    uint32_t W, uint32_t H, uint32_t* err, cudaStream_t st, uint32_t n_img = 1);
cudaError_t backward(const __nv_bfloat16* feat16, const float* label, __nv_bfloat16* const wb[4],
                     const __nv_bfloat16* act1, const __nv_bfloat16* act2,
                     const __nv_bfloat16* act3, const float* prob, __nv_bfloat16* g16, float* g32,
                     __nv_bfloat16* dz_a, __nv_bfloat16* dz_b, float* wpart, float* grads,
                     float* loss_sum, uint32_t W, uint32_t H, uint32_t* err, cudaStream_t st);
// CTAs of the weight-gradient kernels for an image of H rows, and the floats
// of their partial-sum buffer (one row of a layer's gradients per CTA)
int wgrad_blocks(uint32_t H);
size_t wgrad_part_floats(uint32_t H);
cudaError_t adam(float* params, const float* grads, float* m, float* v, uint32_t n, float lr,
                 uint32_t step, cudaStream_t st);
size_t packed_fp8_bytes(int l);
cudaError_t pack_weights_fp8(const float* params, const float* const scale[3], uint8_t* const w8[3],
                             cudaStream_t st);
cudaError_t forward_fp8(const __nv_bfloat16* feat16, const float* params, __nv_bfloat16* const wf[4],
                        uint8_t* const w8[3], const float* const inv[3], const float act_scale[3],
                        uint8_t* act8_1, uint8_t* act8_2, uint8_t* act8_3, float* prob, uint32_t W,
                        uint32_t H, uint32_t* err, cudaStream_t st, uint32_t n_img = 1);
cudaError_t activation_amax(const __nv_bfloat16* const act[3], uint64_t P, unsigned* amax3,
                            cudaStream_t st);
}  // namespace nn

}  // namespace rt

// the opaque scene of the C-ABI
struct rt_scene {
  int device = 0;
  uint32_t ns = 0, nt = 0, n = 0, nm = 0, nl = 0;
  void* block = nullptr;       // persistent device allocation
  float4* nodes = nullptr;
  float4* nodes4 = nullptr;
  float4* nodes_sah = nullptr; // binary tree rebuilt with the SAH over the same leaves (sah.cu)
  uint32_t n4 = 0, n_top = 0;
  bool wide_built = false;     // nodes4 holds the 4-wide tree (built on first use)
  int tree = RT_TREE_SAH;      // the tree renders walk (rt_scene_set_traversal)
  float4* prims = nullptr;
  float4* mats = nullptr;
  float4* lights = nullptr;
  uint64_t* keys = nullptr;
  int32_t* parent = nullptr;
  uint32_t* err = nullptr;
  uint32_t* h_err = nullptr;   // pinned
  float color_scale = 1.f;
  rt::Workspace ws;
};

// error message plumbing and host helpers (rt_api.cu)
void rt_set_error(const std::string& msg);
namespace rt {
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
int ensure_workspace(const rt_scene* sc, uint32_t W, uint32_t H);
int make_render_args(const rt_scene* scene, const rt_camera* cam, float eye_sep, float convergence,
                     uint32_t W, uint32_t H, uint32_t max_depth, RenderArgs& a);
}  // namespace rt
