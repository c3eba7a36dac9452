/*
 * rt_stereo.h -- C-ABI of the GB300 stereo ray tracer.
 *
 * The library computes a stereo pair: two images of one scene seen from two
 * cameras at the observer's eyes (paper Sec. 2: stereoscopic synthesis is
 * the computation of two projections of the scene from two cameras; Sec. 3:
 * the left and right channel are independent -- "parallel level 1" -- and
 * each channel's pixels are traced in parallel -- "parallel level 2").
 * Each pixel is ray traced (Sec. 3, Table 1: reverse/"classical" ray tracing
 * over a BVH): a primary ray, one shadow ray per light facing the surface,
 * and mirror reflection rays up to a fixed depth, shaded to RGB.
 *
 * Conventions shared by every entry point
 *  - Return value: RT_OK (0) or a negative RT_ERR_* code. No C++ exception
 *    crosses this boundary. rt_last_error() gives a message for the calling
 *    thread's last failure.
 *  - "host" pointers are ordinary CPU memory (pageable or pinned); "device"
 *    pointers are CUDA global memory of the current device (for example the
 *    data pointer of a CUDA torch tensor).
 *  - cuda_stream is a cudaStream_t (NULL = legacy default stream). Work is
 *    enqueued on it and the call returns before the GPU finishes, except
 *    where a call says it synchronises. Errors found on the host (bad
 *    arguments, allocation failure) are returned at once; a device-side
 *    check that trips (a traversal or queue bound) is reported by the next
 *    rt_sync_status() on the scene.
 *  - A scene is used by one stream at a time: renders of one scene must not
 *    overlap (they share the scene's scratch buffers).
 *
 * Geometry conventions (the paper fixes none of these; they are readings):
 *  - Right-handed world space. Spheres are (centre, radius); triangles are
 *    (v0, v1, v2) and two-sided. Primitive ids: spheres 0..n_spheres-1, then
 *    triangles n_spheres..n_spheres+n_tris-1; no hit = 0xFFFFFFFF.
 *  - Closest hit = smallest t > 0; equal t resolves to the lower id.
 *  - Camera: off-axis stereo. fwd = normalize(forward), right =
 *    normalize(forward x up), up' = right x fwd. Pixel (i, j) (row 0 = top)
 *    aims at Q = eye + convergence * (fwd + nx right + ny up') with
 *    nx = (2(i+0.5)/W - 1) tan(vfov/2) W/H and ny = (1 - 2(j+0.5)/H) tan(vfov/2).
 *    The left eye sits at eye - (eye_sep/2) right, the right eye at
 *    eye + (eye_sep/2) right; both aim at the same Q, so a point at view
 *    depth z appears f_px * eye_sep * (1/z - 1/convergence) pixels further
 *    right in the left image, f_px = (H/2)/tan(vfov/2).
 *  - Shading (Whitted): at a hit p with normal n facing the ray,
 *    local = albedo * (0.1 + sum over lights with n.l > 0 and an unblocked
 *    shadow ray of intensity * n.l); colour = (1 - r) local + r colour of the
 *    mirror ray while depth < max_depth (the reflected term is 0 at
 *    max_depth); a miss returns the background (0.2, 0.3, 0.5). Secondary
 *    rays start at p + n * 1e-4 * max(1, |p|_inf); a shadow ray towards a
 *    light at distance L is blocked by a hit with t < L - that offset.
 *    Output = colour clamped to [0, 1].
 */
#ifndef RT_STEREO_H
#define RT_STEREO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RT_OK 0
#define RT_ERR_INVALID_ARG (-1)   /* an argument failed validation            */
#define RT_ERR_CUDA (-2)          /* a CUDA runtime call failed                */
#define RT_ERR_OOM (-3)           /* device or host allocation failed          */
#define RT_ERR_TIMEOUT (-4)       /* a device loop hit its iteration bound     */
#define RT_ERR_DEVICE_CHECK (-5)  /* a device-side bound or index check failed */

#define RT_MAX_DEPTH 16
#define RT_MISS_ID 0xFFFFFFFFu

/* Scene records: little-endian, no padding (20, 40, 16, 16, 40 bytes). */
typedef struct { float center[3]; float radius; uint32_t material; } rt_sphere;
typedef struct { float v0[3]; float v1[3]; float v2[3]; uint32_t material; } rt_triangle;
/* albedo in [0,1]^3, reflectivity r in [0,1] */
typedef struct { float albedo[3]; float reflectivity; } rt_material;
/* white point light, no distance falloff */
typedef struct { float position[3]; float intensity; } rt_light;
/* the centre ("cyclopean") eye; vfov_deg is the vertical field of view */
typedef struct { float eye[3]; float forward[3]; float up[3]; float vfov_deg; } rt_camera;

typedef struct rt_scene rt_scene;  /* opaque */

/*
 * rt_scene_create -- upload a scene and build its BVH on the GPU.
 * Paper: Sec. 4 (the host prepares the scene -- objects, polygons, lights --
 * and copies it to GPU memory) and Table 1 (BVH trees as the acceleration
 * structure). The BVH is a linear BVH: FP64 centroid bounds and 10-bit per
 * axis Morton codes, 64-bit keys (morton << 32 | primitive id) sorted on
 * the GPU, a binary radix tree over the keys, FP32 boxes refitted bottom-up
 * (sphere boxes rounded outward).
 *   spheres/tris/mats/lights: host arrays of n_* records; copied, the caller
 *     keeps ownership. n_spheres + n_tris >= 1 and < 2^31; n_mats >= 1;
 *     n_lights >= 1. Every material index < n_mats; radii > 0; all values
 *     finite; reflectivity and albedo in [0, 1]; intensity >= 0.
 *   cuda_stream: stream for the upload and build; the call synchronises it
 *     before returning.
 *   out_scene: receives the new scene; owned by the caller, released with
 *     rt_scene_destroy.
 * Errors: RT_ERR_INVALID_ARG (validation), RT_ERR_OOM, RT_ERR_CUDA.
 */
int rt_scene_create(const rt_sphere* spheres, uint32_t n_spheres,
                    const rt_triangle* tris, uint32_t n_tris,
                    const rt_material* mats, uint32_t n_mats,
                    const rt_light* lights, uint32_t n_lights,
                    void* cuda_stream, rt_scene** out_scene);

/* Release a scene and all device memory it owns. NULL is ignored. The
 * caller must make sure no work using the scene is still in flight. */
void rt_scene_destroy(rt_scene* scene);

/*
 * rt_render_stereo -- trace both eyes of one stereo pair.
 * Paper: Sec. 2-3 (two projections from two eye cameras; left and right
 * channel computed in parallel; per-pixel ray tracing within a channel).
 *   cam: host pointer; forward x up must not vanish; 0 < vfov_deg < 180.
 *   eye_sep >= 0: distance between the eyes. convergence > 0: distance of the
 *     shared image window (zero-disparity plane) along forward.
 *   W, H >= 1 pixels per eye, 2*W*H <= 2^31; max_depth <= RT_MAX_DEPTH
 *     reflection bounces after the primary hit.
 *   out_L, out_R: device buffers of H*W*3 float32 each, row-major, row 0 at
 *     the top, RGB interleaved; owned by the caller; fully overwritten.
 *   cuda_stream: the stream the render is enqueued on (asynchronous).
 * The first render at a new size may allocate scene-owned scratch (which is
 * then reused); it does not synchronise.
 * Errors: RT_ERR_INVALID_ARG, RT_ERR_OOM, RT_ERR_CUDA on the host;
 * device-side bounds are reported by rt_sync_status.
 */
int rt_render_stereo(const rt_scene* scene, const rt_camera* cam,
                     float eye_sep, float convergence,
                     uint32_t W, uint32_t H, uint32_t max_depth,
                     float* out_L, float* out_R, void* cuda_stream);

/*
 * rt_render_stereo_aux -- rt_render_stereo plus per-pixel and per-ray-kind
 * diagnostics, for tests and measurement. Any of the extra pointers may be
 * NULL. All are device pointers owned by the caller:
 *   hit_id_L/R: H*W uint32, primary-ray hit primitive id (RT_MISS_ID on miss)
 *   depth_L/R:  H*W float32, view depth of the primary hit (t * d.fwd),
 *               +infinity on a miss
 *   ray_counts: 3 uint64: rays traced by kind (primary, shadow, reflection)
 *   work:       9 uint64: per kind (primary, shadow, reflection) the internal
 *               BVH nodes visited, ray-sphere tests, ray-triangle tests. When
 *               non-NULL the instrumented traversal variant runs (slower).
 */
int rt_render_stereo_aux(const rt_scene* scene, const rt_camera* cam,
                         float eye_sep, float convergence,
                         uint32_t W, uint32_t H, uint32_t max_depth,
                         float* out_L, float* out_R,
                         uint32_t* hit_id_L, uint32_t* hit_id_R,
                         float* depth_L, float* depth_R,
                         uint64_t* ray_counts, uint64_t* work,
                         void* cuda_stream);

/*
 * rt_render_stereo_rows -- a horizontal band of both eyes of a stereo pair.
 * Paper: Sec. 3, Figure 1 (the image is divided into parts and each
 * processor renders its part); with several GPUs, each renders one band of
 * rows of both eyes over its own copy of the scene. The rays are those of
 * the whole W x H pair: the rows row0 .. row0 + n_rows - 1 of the band equal
 * the same rows of rt_render_stereo bit for bit, so bands stitched in row
 * order give the full pair.
 *   W, H: the whole image; 1 <= n_rows, row0 + n_rows <= H.
 *   out_L, out_R: DEVICE buffers of n_rows*W*3 float32 each, row-major
 *     (band row 0 = image row row0); owned by the caller.
 *   ray_counts: DEVICE 3 uint64 or NULL (rays of the band by kind).
 * Otherwise as rt_render_stereo (asynchronous on cuda_stream).
 */
int rt_render_stereo_rows(const rt_scene* scene, const rt_camera* cam,
                          float eye_sep, float convergence,
                          uint32_t W, uint32_t H, uint32_t max_depth,
                          uint32_t row0, uint32_t n_rows,
                          float* out_L, float* out_R, uint64_t* ray_counts,
                          void* cuda_stream);

/*
 * rt_render_stereo_host -- end-to-end render into HOST buffers.
 * Paper: Sec. 4-5 (the synthesis time splits into GPU computation and the
 * copies between CPU and GPU memory). Both images land in host_L/host_R
 * (H*W*3 float32 each, same layout) and the stream is synchronised before
 * returning. Pinned host buffers that the GPU can address (cudaHostAlloc /
 * pinned torch tensors) are written directly by the final kernel over the
 * CPU-GPU link; other host memory is filled by a copy from scene-owned
 * device frames.
 */
int rt_render_stereo_host(const rt_scene* scene, const rt_camera* cam,
                          float eye_sep, float convergence,
                          uint32_t W, uint32_t H, uint32_t max_depth,
                          float* host_L, float* host_R, void* cuda_stream);

/*
 * rt_render_stereo_sequence -- n_frames stereo pairs of one scene into HOST
 * buffers, the device-to-host copy of each pair overlapped with the
 * rendering of the next. Paper: Sec. 4-5 (a frame's synthesis time splits
 * into GPU computation and CPU-GPU transfer; Figure 7); overlapping the two
 * hides the transfer behind the computation of the following frame.
 *   cams[n_frames]:  one camera per frame (host array); eye_sep,
 *                    convergence, W, H and max_depth as in rt_render_stereo
 *                    and shared by all frames
 *   host_L[f], host_R[f]: frame f's images, H*W*3 float32 each (host
 *                    memory; pinned memory lets the copies run
 *                    asynchronously). The same buffer may be named for
 *                    several frames: copies run in frame order, so it ends
 *                    up holding the last of them.
 * Each pair is rendered on cuda_stream into one of two scene-owned device
 * frame slots and copied out on a scene-owned copy stream (the slot is not
 * reused before its copy has finished). Returns when every image is in host
 * memory. Every camera is validated before any work is queued.
 * Errors: RT_ERR_INVALID_ARG (as rt_render_stereo, or a NULL camera array,
 * pointer array or buffer), RT_ERR_OOM, RT_ERR_CUDA.
 */
int rt_render_stereo_sequence(const rt_scene* scene, const rt_camera* cams, uint32_t n_frames,
                              float eye_sep, float convergence,
                              uint32_t W, uint32_t H, uint32_t max_depth,
                              float* const* host_L, float* const* host_R,
                              void* cuda_stream);

/*
 * rt_sync_status -- synchronise cuda_stream and report device-side checks
 * raised by earlier work on the scene (then clear them).
 * Returns RT_OK, RT_ERR_TIMEOUT (a traversal or queue loop reached its
 * iteration bound), RT_ERR_DEVICE_CHECK (a stack, queue or index bound was
 * exceeded) or RT_ERR_CUDA.
 */
int rt_sync_status(const rt_scene* scene, void* cuda_stream);

/*
 * rt_scene_get_bvh -- copy the scene's LBVH to HOST arrays (test hook;
 * synchronises). n = number of primitives. Any pointer may be NULL.
 *   keys[n]:        sorted 64-bit keys (morton30 << 32 | primitive id)
 *   left[n-1], right[n-1]: children of internal node i (binary radix tree
 *                   numbering, root 0): >= 0 internal node, < 0 leaf ~k
 *                   (leaf k holds the primitive of keys[k])
 *   parent[2n-1]:   parent of internal node i at [i], of leaf k at [n-1+k];
 *                   -1 for the root
 *   inner_box[(n-1)*6], leaf_box[n*6]: FP32 boxes, lo xyz then hi xyz
 */
int rt_scene_get_bvh(const rt_scene* scene, uint64_t* keys, int32_t* left, int32_t* right,
                     int32_t* parent, float* inner_box, float* leaf_box);

/*
 * rt_debug_set_node -- TEST HOOK; the paper has no counterpart. Overwrites
 * the children of internal node `node` with (left, right) (>= 0 internal
 * node < n-1, < 0 leaf ~k with k < n; out-of-range values are rejected with
 * RT_ERR_INVALID_ARG) and, when empty_right != 0, gives the right child an
 * empty box. It lets a test build a cycle in the BVH (for example node 0 as
 * its own left child with an empty right child) to check that traversal
 * stops at its iteration bound and rt_sync_status reports RT_ERR_TIMEOUT;
 * every index stays in range, so no memory outside the scene is touched.
 * It edits the LBVH (renders walk it after
 * rt_scene_set_traversal(scene, RT_TREE_LBVH)). Synchronises the device.
 */
int rt_debug_set_node(rt_scene* scene, uint32_t node, int32_t left, int32_t right,
                      int empty_right);

/*
 * rt_debug_get_sah_tree -- TEST HOOK. Copies the scene's SAH render tree (the
 * tree RT_TREE_SAH renders walk, rebuilt from the LBVH's leaves) to the HOST
 * array nodes[(n-1)*16] (n = primitives; nothing is copied when n == 1): per
 * inner node (root 0) 16 words, the FP32 child boxes as lo.x, hi.x, lo.y, hi.y
 * of child 0, the same of child 1, lo.z, hi.z of child 0, lo.z, hi.z of child
 * 1, then the two children as int32 bit patterns (>= 0 inner node, < 0 leaf
 * ~k, k indexing the LBVH's sorted primitives) and two unused words.
 * Synchronises the device. RT_ERR_INVALID_ARG for a NULL scene or nodes.
 */
int rt_debug_get_sah_tree(const rt_scene* scene, float* nodes);

/*
 * rt_debug_set_sah_slicing -- TEST HOOK. Process-wide: with enable != 0 (the
 * default) scene creation builds the top levels of the SAH tree (levels of at
 * most 32 nodes averaging at least 16384 leaves) with every node sliced over
 * many blocks; with 0 every level runs one block per node. Both give the same
 * tree; the switch lets a test compare them. Host-only; affects scenes
 * created afterwards. Returns RT_OK.
 */
int rt_debug_set_sah_slicing(int enable);

/*
 * rt_debug_set_pool_capacity -- TEST HOOK; the paper has no counterpart.
 * Limits the two drain pools of the scene's renders to `entries` rays each
 * (0 restores the full capacity, which is 128 rays per warp of the render
 * kernel; larger values are clamped to it). Once every primary tile has been
 * handed out, the render kernel's warps hand their queued shadow and mirror
 * rays to these pools and take them back in batches of 32; rays that do not
 * fit stay with the warp that queued them. A small capacity forces that
 * fallback (and the empty entries it publishes at the end of a pool), which
 * must render the same image bit for bit. Returns RT_ERR_INVALID_ARG for a
 * NULL scene. Host-only; takes effect with the next render.
 */
int rt_debug_set_pool_capacity(rt_scene* scene, uint32_t entries);

/*
 * rt_scene_set_traversal -- choose the tree renders of this scene walk
 * (Table 1 of the paper: BVH trees). Every scene holds three over the same
 * leaves (one primitive each) and the same conservative leaf boxes, so all
 * three give the same images bit for bit:
 *   RT_TREE_SAH  (0, default) a binary tree rebuilt on the GPU from the
 *                LBVH's leaves with the surface area heuristic over binned
 *                centroids; on the 256k-triangle blob scene at 1080p it needs
 *                15 % fewer node visits for shadow and mirror rays than the
 *                LBVH and is the fastest walk on GB300;
 *   RT_TREE_WIDE (1) the 4-wide tree collapsed from the SAH tree (every
 *                inner node at even depth holds its grandchildren; its top
 *                two levels staged in shared memory);
 *   RT_TREE_LBVH (2) the Morton-code binary radix tree itself, the tree
 *                rt_scene_get_bvh returns and rt_debug_set_node edits.
 * The instrumented work counts of rt_render_stereo_aux follow the binary
 * tree in use (the SAH tree for RT_TREE_WIDE). The 4-wide tree is built the
 * first time it is chosen (synchronous: the device is synchronised and a
 * scratch buffer of ~21 bytes per primitive is allocated and freed; errors
 * RT_ERR_CUDA); choosing a tree is otherwise host-only and takes effect with
 * the next render. Other values: RT_ERR_INVALID_ARG.
 */
#define RT_TREE_SAH 0
#define RT_TREE_WIDE 1
#define RT_TREE_LBVH 2
int rt_scene_set_traversal(rt_scene* scene, int tree);

/*
 * rt_profile_enable / rt_profile_read -- per-stage GPU time of the last
 * render of a scene (paper Sec. 4, Figure 7: time spent on the basic
 * procedures of the synthesis). While enabled, every render records a CUDA
 * event on its stream after each stage. rt_profile_read waits for the last
 * render's events and writes RT_NUM_STAGES floats (milliseconds) to the
 * HOST array ms: [0] clears, [1] ray tracing (primary, shadow and mirror
 * rays, one persistent kernel), [2] resolve to float RGB, and for
 * rt_render_stereo_reproj [3] forward warp, [4] retrace network, [5] retrace
 * mask, [6] tracing the masked right pixels, [7] right-image composition
 * (stages a call does not run read 0).
 * Returns RT_ERR_INVALID_ARG if profiling was off during the last render.
 */
#define RT_NUM_STAGES 8
int rt_profile_enable(rt_scene* scene, int on);
int rt_profile_read(const rt_scene* scene, float* ms);

/*
 * rt_build_lbvh_noalloc -- the LBVH build of rt_scene_create, for callers
 * that cannot allocate device memory. The paper has no counterpart: this
 * entry point exists for code that must not call cudaMalloc, such as a
 * plugin whose host application hands out all GPU memory from its own pool,
 * or a real-time loop that cannot afford cudaMalloc's implicit device
 * synchronisation. It runs the same kernels as rt_scene_create but writes
 * into the caller's buffers and keeps its scratch in a static device array
 * of 13 MiB that every GPU loading this library holds until the process
 * exits; nothing is allocated.
 *   d_spheres / d_tris: DEVICE arrays of n_spheres rt_sphere and n_tris
 *     rt_triangle records (not validated: the caller vouches for finite
 *     values and material indices).
 *   1 <= n_spheres + n_tris <= 1,048,576 (2^20); larger builds are
 *     rejected with RT_ERR_INVALID_ARG.
 *   Outputs (DEVICE, caller-owned, d_nodes and d_prims 16-byte aligned):
 *     d_nodes:  max(n-1,1) nodes of 16 floats (64 B): child boxes and child
 *               indices in the layout the renderer reads;
 *     d_prims:  n leaf records of 12 floats (48 B);
 *     d_keys:   n sorted keys; d_parent: 2n-1 parent indices (as in
 *               rt_scene_get_bvh).
 *   The call synchronises cuda_stream and returns RT_ERR_DEVICE_CHECK if the
 *   device-side refit check trips. Every call uses the same scratch array:
 *   calls whose GPU work overlaps (other streams or host threads) race and
 *   must be serialised by the caller. Each call looks up the array's device
 *   address in the current context (cudaGetSymbolAddress), so the address
 *   stays right after a device reset or a context switch.
 */
int rt_build_lbvh_noalloc(const rt_sphere* d_spheres, uint32_t n_spheres,
                          const rt_triangle* d_tris, uint32_t n_tris,
                          float* d_nodes, float* d_prims, uint64_t* d_keys, int32_t* d_parent,
                          void* cuda_stream);

/* ------------------------------------------------------------------------
 * Learned right-eye reprojection. The paper computes the left and right
 * channel independently (Sec. 3, "parallel level 1"); this extension traces
 * the left channel, warps it to the right eye, and re-traces only the right
 * pixels that a small network (or a disocclusion) marks. The full right-eye
 * trace stays the reference it is judged against.
 *
 * Network: 3x3 convolutions 10 -> 32 -> 32 -> 32 -> 1, zero padding 1,
 * ReLU, sigmoid; BF16 operands on the tensor cores, FP32 accumulation,
 * FP32 master weights. Parameters (RT_NET_PARAMS floats) in this order:
 * W1[32][10][3][3], b1[32], W2[32][32][3][3], b2[32], W3[32][32][3][3],
 * b3[32], W4[1][32][3][3], b4[1].
 * Features of a right pixel (BF16, 16 channels per pixel, channels 10-15
 * zero; all zero on a hole): min(z/100, 1), the normal (3), hash(hit id) =
 * (fmix32(id) >> 8) * 2^-24 (MurmurHash3 finaliser), the left RGB (3), the
 * disparity / 16 and the reflectivity of the hit surface (mirror pixels
 * change colour with the viewpoint, so a warp cannot carry them), taken
 * from the left pixel that the forward warp puts there: a left pixel (i, j) at view depth z lands on column
 * floor(i - D + 0.5) of row j, D = f_px * eye_sep * (1/z - 1/convergence),
 * f_px = (H/2)/tan(vfov/2); the nearest z wins, equal z the lower index.
 * A left pixel whose ray missed is a source at infinity (z = +inf, zero
 * normal, background colour), so only disocclusions and the uncovered
 * border remain holes.
 */
#define RT_NET_PARAMS 21697
typedef struct rt_net rt_net;  /* opaque */

/* Upload RT_NET_PARAMS host floats (finite) into a new network; synchronises.
 * Errors: RT_ERR_INVALID_ARG, RT_ERR_OOM, RT_ERR_CUDA. */
int rt_net_create(const float* host_params, uint32_t n_params, rt_net** out);
void rt_net_destroy(rt_net* net);
/* Copy the current FP32 parameters to host memory (synchronises). */
int rt_net_get_params(const rt_net* net, float* host_params);
/* Synchronise the stream and report a tensor-core wait that reached its
 * bound in earlier network work (RT_ERR_TIMEOUT), then clear it. */
int rt_net_status(const rt_net* net, void* cuda_stream);

/*
 * rt_net_set_fp8 -- run the network's inference in FP8 from now on
 * (rt_net_forward and rt_render_stereo_reproj; training stays BF16).
 * Layer 1 keeps BF16 operands; its output and the later hidden activations
 * are stored as OCP FP8 E4M3 of (activation * act_scales[i]), i = 0, 1, 2
 * for the outputs of layers 1-3, rounded to nearest even and saturated at
 * +-448. Layers 2-4 multiply E4M3 operands on the tensor cores
 * (tcgen05 kind::f8f6f4, FP32 accumulation) with E4M3 weights scaled per
 * output channel by the largest power of two s with max|w| * s <= 448; the
 * epilogue undoes both scales exactly before the bias.
 *   act_scales: host float[3], each a power of two in [2^-30, 2^30] (see
 *     rt_net_activation_amax for choosing them), or NULL to return to BF16.
 * Packs the current parameters (call it again after training); synchronises.
 * Errors: RT_ERR_INVALID_ARG, RT_ERR_CUDA.
 */
int rt_net_set_fp8(rt_net* net, const float* act_scales);

/*
 * rt_net_activation_amax -- run the BF16 network on a feature map (layout as
 * for rt_net_forward) and return the largest value of each of its three
 * hidden activations (after ReLU) in host_amax[3]; synchronises cuda_stream.
 * A natural FP8 scale for activation i is the largest power of two s with
 * host_amax[i] * s <= 448.
 */
int rt_net_activation_amax(rt_net* net, const uint16_t* d_feat16, uint32_t W, uint32_t H,
                           float* host_amax, void* cuda_stream);

/*
 * rt_net_calibrate_fp8 -- choose the FP8 activation scales from data and
 * switch the network to FP8 inference. The paper has no network; the scales
 * follow the scaling described at rt_net_set_fp8: the BF16 network runs on
 * every feature map, amax[i] is the largest value hidden activation i takes
 * over all of them, and act_scales[i] is the largest power of two s with
 * amax[i] * s <= 448 (the largest E4M3 value; 1 when amax[i] is 0), clamped
 * to [2^-30, 2^30]. Then it does what rt_net_set_fp8(net, act_scales) does.
 *   d_feats: HOST array of n_maps >= 1 DEVICE feature maps, each W*H*16 BF16
 *     (as for rt_net_forward, 16-byte aligned).
 *   host_amax, host_scales: HOST float[3] each, may be NULL; receive the
 *     maxima and the chosen scales.
 * Synchronises cuda_stream. Errors: RT_ERR_INVALID_ARG, RT_ERR_OOM,
 * RT_ERR_CUDA.
 */
int rt_net_calibrate_fp8(rt_net* net, const uint16_t* const* d_feats, uint32_t n_maps, uint32_t W,
                         uint32_t H, float* host_amax, float* host_scales, void* cuda_stream);

/*
 * rt_net_save / rt_net_load -- a training checkpoint in a file: the FP32
 * parameters, both Adam moment vectors and the Adam step count, and the FP8
 * inference state (on/off and the activation scales), so that training
 * continued from a loaded checkpoint performs exactly the updates the saved
 * network would have (training steps are deterministic). The paper has no
 * network; this serves the training loop above.
 * File layout (little-endian, no padding): char magic[8] = "RTNETCK1";
 * uint32 version (1), n_params (RT_NET_PARAMS), adam_step, fp8 (0 or 1);
 * float act_scales[3]; float params[n_params], adam_m[n_params],
 * adam_v[n_params]; uint32 CRC-32 (zlib convention) of all bytes before it.
 *   rt_net_save: path is a HOST file name, created or overwritten. The net
 *     is synchronised with the device first.
 *   rt_net_load: verifies magic, version, size and CRC, then creates a new
 *     network (released with rt_net_destroy) in *out. Synchronises.
 * Errors: RT_ERR_INVALID_ARG (file missing, unreadable, unwritable,
 * truncated or corrupt), RT_ERR_OOM, RT_ERR_CUDA.
 */
int rt_net_save(const rt_net* net, const char* path);
int rt_net_load(const char* path, rt_net** out);

/*
 * rt_net_forward -- retrace probability of every pixel of a W x H feature map.
 *   d_feat16: DEVICE, W*H*16 BF16 (as uint16 bits), row-major pixels,
 *             16-byte aligned (it is read by the tensor-memory-access engine;
 *             a misaligned pointer gives RT_ERR_CUDA).
 *   d_prob:   DEVICE, W*H float32 output in (0, 1).
 * Asynchronous on cuda_stream; the network's activation buffers are grown
 * on demand (allocation on the first call at a size).
 */
int rt_net_forward(rt_net* net, const uint16_t* d_feat16, uint32_t W, uint32_t H, float* d_prob,
                   void* cuda_stream);

/*
 * rt_net_forward_images -- rt_net_forward of n_img feature maps of W x H
 * pixels stored one after the other (d_feat16: n_img*W*H*16 BF16; d_prob:
 * n_img*W*H floats), one launch per layer for all of them. Each image is
 * convolved on its own (zero padding at its borders), so image i's output
 * equals rt_net_forward on image i alone bit for bit. The paper has no
 * network; this serves the multi-frame reprojection below.
 */
int rt_net_forward_images(rt_net* net, const uint16_t* d_feat16, uint32_t n_img, uint32_t W,
                          uint32_t H, float* d_prob, void* cuda_stream);

/*
 * rt_net_train_step -- one step on the mean binary cross-entropy of the
 * network's output against d_label (DEVICE, W*H floats in {0,1}): forward,
 * backward (data gradients on the tensor cores, weight gradients in FP32),
 * then Adam (beta 0.9 / 0.999, eps 1e-8, step size lr) when lr > 0.
 *   host_loss: if non-NULL receives the loss before the update (synchronises).
 *   d_grads:   if non-NULL, DEVICE RT_NET_PARAMS floats receive the gradient.
 */
int rt_net_train_step(rt_net* net, const uint16_t* d_feat16, const float* d_label, uint32_t W,
                      uint32_t H, float lr, float* host_loss, float* d_grads, void* cuda_stream);

/*
 * rt_reproj_warp -- forward warp of a left G-buffer to the right eye.
 *   inputs (DEVICE, W*H pixels each): d_depth_L view depth (+inf = the ray
 *   missed: a source at infinity; <= 0 or NaN: skipped),
 *   d_normal_L (3 floats), d_id_L (hit id), d_rgb_L (3 floats),
 *   d_refl_L (reflectivity of the hit surface, 0 on a miss; may be NULL:
 *   all 0).
 *   d_zbuf: DEVICE scratch of W*H uint64 (overwritten).
 *   outputs (DEVICE, any may be NULL): d_feat16 (W*H*16 BF16 bits),
 *   d_feat32 (W*H*10 floats, the same features before BF16 rounding),
 *   d_hole (W*H bytes: 1 where no left pixel lands, 2 where the left pixel
 *   that lands there hit a reflective surface (reflectivity > 0), else 0),
 *   d_warped (W*H*3 floats).
 */
int rt_reproj_warp(const float* d_depth_L, const float* d_normal_L, const uint32_t* d_id_L,
                   const float* d_rgb_L, const float* d_refl_L, uint32_t W, uint32_t H, float f_px,
                   float eye_sep,
                   float convergence, uint64_t* d_zbuf, uint16_t* d_feat16, float* d_feat32,
                   uint8_t* d_hole, float* d_warped, void* cuda_stream);

/*
 * rt_reproj_training_pair -- one training example: traces both eyes in full
 * (d_out_L, d_out_R as in rt_render_stereo), warps the left eye, writes the
 * right-eye features (d_feat16) and labels d_label = 1 where the pixel is a
 * hole or some channel of the warped colour differs from the full trace by
 * more than label_threshold (DEVICE buffers of W*H*16 BF16 / W*H floats).
 */
int rt_reproj_training_pair(const rt_scene* scene, const rt_camera* cam, float eye_sep,
                            float convergence, uint32_t W, uint32_t H, uint32_t max_depth,
                            float* d_out_L, float* d_out_R, uint16_t* d_feat16, float* d_label,
                            float label_threshold, void* cuda_stream);

/*
 * rt_render_stereo_reproj -- a stereo pair with the right eye reprojected:
 * traces the left eye (out_L exactly as rt_render_stereo), warps it to the
 * right grid, runs the network (net may be NULL: no network), traces the
 * right pixels that are holes, that show a reflective surface (a mirror's
 * colour depends on the viewpoint, so the warp cannot carry it) or whose
 * retrace probability p exceeds threshold, and writes out_R = traced
 * colour there, warped colour elsewhere. d_n_retraced (DEVICE uint32, may be
 * NULL) receives the number of retraced right pixels. Asynchronous.
 */
int rt_render_stereo_reproj(const rt_scene* scene, const rt_camera* cam, float eye_sep,
                            float convergence, uint32_t W, uint32_t H, uint32_t max_depth,
                            rt_net* net, float threshold, float* d_out_L, float* d_out_R,
                            uint32_t* d_n_retraced, void* cuda_stream);

/*
 * rt_render_stereo_reproj_frames -- rt_render_stereo_reproj for up to
 * RT_MAX_FRAMES frames of one scene in one pass: each stage runs once for
 * all frames (one launch traces the left eyes of every frame, one warps
 * them, one per network layer classifies every right pixel, one retraces
 * the masked right pixels of every frame, one composes). Frame f's images
 * equal those of rt_render_stereo_reproj with cams[f] bit for bit.
 *   cams: HOST array of n_frames cameras (1 <= n_frames <= RT_MAX_FRAMES),
 *     all with the same vfov_deg (the warp needs one focal length).
 *   d_out_L, d_out_R: DEVICE, n_frames*H*W*3 float32 each, frame after frame
 *     (each frame laid out as rt_render_stereo's images).
 *   d_n_retraced: DEVICE uint32 or NULL: right pixels retraced, all frames.
 * Otherwise as rt_render_stereo_reproj (asynchronous on cuda_stream).
 */
#define RT_MAX_FRAMES 8
int rt_render_stereo_reproj_frames(const rt_scene* scene, const rt_camera* cams, uint32_t n_frames,
                                   float eye_sep, float convergence, uint32_t W, uint32_t H,
                                   uint32_t max_depth, rt_net* net, float threshold, float* d_out_L,
                                   float* d_out_R, uint32_t* d_n_retraced, void* cuda_stream);

/*
 * rt_stereo_composite -- convert a stereo pair into a display frame.
 * Paper Sec. 3: GPU post-processing turns the stereo pair into the frame
 * format of the display device, e.g. an anaglyph.
 *   d_L, d_R: DEVICE, H*W*3 float32 each (as written by rt_render_stereo).
 *   mode RT_COMPOSITE_ANAGLYPH_COLOR: out = (L.r, R.g, R.b) per pixel;
 *   mode RT_COMPOSITE_ANAGLYPH_GRAY:  out = (y(L), y(R), y(R)) with
 *        y = fma(0.114, b, fma(0.587, g, 0.299 r)) in FP32;
 *   mode RT_COMPOSITE_SIDE_BY_SIDE:   out = H rows of 2W pixels, left eye first.
 *   d_out: DEVICE, H*W*3 floats (H*2W*3 side by side), caller-owned.
 * Asynchronous on cuda_stream. Errors: RT_ERR_INVALID_ARG, RT_ERR_CUDA.
 */
#define RT_COMPOSITE_ANAGLYPH_COLOR 0
#define RT_COMPOSITE_ANAGLYPH_GRAY 1
#define RT_COMPOSITE_SIDE_BY_SIDE 2
int rt_stereo_composite(const float* d_L, const float* d_R, uint32_t W, uint32_t H, int mode,
                        float* d_out, void* cuda_stream);

/*
 * Batched stereo rendering: many stereo requests of uneven resolutions,
 * depths and scenes traced by ONE persistent kernel launch, replayed from a
 * captured CUDA graph. Paper Sec. 3 splits the image over parallel workers
 * (Figure 1) and Sec. 4 / Figure 8 studies how the CUDA launch shape ("network
 * size") affects the time; here every tile of every request is one unit of a
 * shared work list, and the launch shape (tile shape, resident blocks per SM,
 * mirror-queue capacity, request order) is chosen by a measured autotuner.
 * Each request's images equal, bit for bit, what rt_render_stereo gives for
 * the same scene and arguments.
 *
 * rt_request (88 bytes, little-endian, naturally aligned):
 *   scene       a scene from rt_scene_create; it must outlive the batch and
 *               must not be rendered by another call while a launch of the
 *               batch is in flight (the batch reads its BVH, not its scratch)
 *   camera, eye_sep, convergence, W, H, max_depth   as for rt_render_stereo
 *   reserved    must be 0
 *   d_out_L, d_out_R   DEVICE, H*W*3 float32 each, caller-owned
 * Limits: 1 <= n_requests <= RT_BATCH_MAX_REQUESTS; sum of 2*W*H over the
 * requests < 2^32; every request as rt_render_stereo validates it.
 *
 * rt_batch_config (24 bytes):
 *   tile_w x tile_h   pixels per 32-ray tile: 16 pixels traced for both eyes,
 *                     the two rays of a pixel in neighbouring lanes ((2,8),
 *                     (4,4), (8,2) or (16,1)), or 32 pixels of one eye ((4,8),
 *                     (8,4), (16,2) or (32,1))
 *   blocks_per_sm     resident blocks of 128 threads per SM, 1..the kernel's
 *                     occupancy limit (0 = that limit)
 *   cap_r             mirror-queue entries per warp: 64, 128 or 256
 *   order             tile order over requests: RT_BATCH_ORDER_GIVEN,
 *                     RT_BATCH_ORDER_LARGEST_FIRST, RT_BATCH_ORDER_SMALLEST_FIRST
 *   track_latency     1 = record per request the device time at which its
 *                     last ray finished (read with rt_batch_stats)
 */
#define RT_BATCH_MAX_REQUESTS 4096
#define RT_BATCH_ORDER_GIVEN 0
#define RT_BATCH_ORDER_LARGEST_FIRST 1
#define RT_BATCH_ORDER_SMALLEST_FIRST 2
typedef struct {
  const rt_scene* scene;
  rt_camera camera;
  float eye_sep, convergence;
  uint32_t W, H, max_depth, reserved;
  float* d_out_L;
  float* d_out_R;
} rt_request;
typedef struct {
  uint32_t tile_w, tile_h, blocks_per_sm, cap_r, order, track_latency;
} rt_batch_config;
typedef struct rt_batch rt_batch;  /* opaque */

/*
 * rt_batch_create -- validate the requests, allocate the batch's device
 * memory (colour sums for every pixel of every request, per-warp ray queues,
 * the request table) and capture the launch sequence (request-table upload,
 * clears, the persistent render kernel, the resolve kernel) into a CUDA
 * graph.
 *   reqs: host array of n_requests records (copied).
 *   cfg:  host pointer or NULL (= tile 4x4, occupancy limit, cap_r 64,
 *         largest request first, latency tracking on).
 *   out_batch: receives the batch; released with rt_batch_destroy.
 * Synchronous. Errors: RT_ERR_INVALID_ARG, RT_ERR_OOM, RT_ERR_CUDA.
 */
int rt_batch_create(const rt_request* reqs, uint32_t n_requests, const rt_batch_config* cfg,
                    rt_batch** out_batch);

/* Release the batch (waits for its last launch). NULL is ignored. */
void rt_batch_destroy(rt_batch* batch);

/*
 * rt_batch_launch -- replay the batch's graph on cuda_stream: every request
 * is traced and its two images written. Asynchronous; a device-side check
 * that trips is reported by rt_batch_stats. Launches of one batch must not
 * overlap each other.
 */
int rt_batch_launch(rt_batch* batch, void* cuda_stream);

/*
 * rt_batch_set_camera -- change request i's camera, eye_sep and convergence
 * for the following launches (the graph uploads the request table from
 * pinned host memory each launch). Waits for the previous launch to finish
 * before editing that table. Errors: RT_ERR_INVALID_ARG.
 */
int rt_batch_set_camera(rt_batch* batch, uint32_t i, const rt_camera* cam, float eye_sep,
                        float convergence);

/*
 * rt_batch_autotune -- time candidate configurations of this batch with CUDA
 * events on cuda_stream (each: one warm-up launch, then `reps` timed
 * launches, median) by coordinate descent over tile shape, blocks per SM,
 * mirror-queue capacity and request order, starting from the current
 * configuration; keep the fastest and re-capture the graph with it.
 *   chosen: host, receives the configuration kept (may be NULL).
 *   best_ms: host, receives its median launch time in ms (may be NULL).
 * Synchronous; the request outputs hold the last candidate's (identical)
 * images. Errors: RT_ERR_INVALID_ARG, RT_ERR_CUDA, RT_ERR_OOM, and the
 * device-check codes of rt_batch_stats.
 */
int rt_batch_autotune(rt_batch* batch, uint32_t reps, void* cuda_stream, rt_batch_config* chosen,
                      float* best_ms);

/*
 * rt_batch_stats -- wait for the batch's last launch and report it.
 *   ray_counts: host uint64[3] or NULL: primary, shadow and mirror rays of
 *     the last launch, all requests together.
 *   request_ms: host float[n_requests] or NULL: per request, the time from
 *     the start of the render kernel to the completion of its last ray
 *     (needs track_latency; else filled with -1).
 *   cfg: host or NULL: the configuration in use.
 * Errors: RT_ERR_TIMEOUT / RT_ERR_DEVICE_CHECK if a device bound tripped in
 * the last launch, RT_ERR_CUDA.
 */
int rt_batch_stats(rt_batch* batch, uint64_t* ray_counts, float* request_ms, rt_batch_config* cfg);

/* Number of primitives of the scene (0 for NULL). */
uint32_t rt_scene_num_prims(const rt_scene* scene);

/* Message of the calling thread's last failure ("" if none). */
const char* rt_last_error(void);

/* Library version string. */
const char* rt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RT_STEREO_H */
