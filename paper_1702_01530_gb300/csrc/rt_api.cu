// C-ABI entry points of the stereo ray tracer (declared in include/rt_stereo.h).
//
// Host-side duties only: argument validation, device memory ownership, the
// stereo camera basis (computed in FP64 once per call), and status
// reporting. Every step of the rendering itself runs in the CUDA kernels of
// lbvh.cu and trace.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rt_internal.cuh"

static thread_local std::string g_last_error;

void rt_set_error(const std::string& msg) { g_last_error = msg; }

namespace rt {

int fail(int code, const std::string& msg) {
  rt_set_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace rt

using rt::cuda_fail;
using rt::fail;

namespace {

bool finite3(const float* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

void free_workspace(rt::Workspace& ws) {
  if (ws.seq_copy) cudaStreamSynchronize(ws.seq_copy);
  if (ws.base) cudaFree(ws.base);
  if (ws.frame) cudaFree(ws.frame);
  if (ws.seq_frame) cudaFree(ws.seq_frame);
  for (int k = 0; k < 2; ++k) {
    if (ws.seq_rendered[k]) cudaEventDestroy(ws.seq_rendered[k]);
    if (ws.seq_copied[k]) cudaEventDestroy(ws.seq_copied[k]);
  }
  if (ws.seq_copy) cudaStreamDestroy(ws.seq_copy);
  if (ws.rp.base) cudaFree(ws.rp.base);
  for (cudaEvent_t& e : ws.ev)
    if (e) cudaEventDestroy(e);
  ws = rt::Workspace();
}

}  // namespace

namespace rt {
// grow the scene's scratch to hold a W x H stereo pair with L lights:
// fixed-point accumulators for both eyes and, per resident warp of the
// render kernel, a shadow queue of 32 L + 32 and a mirror queue of 64
// entries (48 B each)
int ensure_workspace(const rt_scene* sc_c, uint32_t W, uint32_t H) {
  rt_scene* sc = const_cast<rt_scene*>(sc_c);
  rt::Workspace& ws = sc->ws;
  const uint64_t pixels = 2ull * W * H;
  const uint64_t n_warps = (uint64_t)rt::render_grid() * (rt::render_threads() / 32);
  const uint32_t cap_s = 32u * sc->nl + 32u, cap_r = 64u;
  if (ws.base && ws.cap_pixels >= pixels && ws.L == sc->nl && ws.n_warps >= n_warps) return RT_OK;
  const uint64_t cap_pixels = ws.cap_pixels > pixels ? ws.cap_pixels : pixels;
  // drain pools: 128 entries per warp and kind (a full pool only makes the
  // warps that cannot hand over their leftovers trace them themselves)
  const uint64_t cap_p = n_warps * 128u;
  size_t b_acc = align256(cap_pixels * 3 * sizeof(uint32_t));
  size_t b_q = align256(n_warps * (cap_s + cap_r) * 3 * sizeof(float4));
  size_t b_p = align256(2 * cap_p * 3 * sizeof(float4));
  size_t b_f = align256(2 * cap_p * sizeof(uint32_t));
  size_t b_c = align256(rt::C_TOTAL * sizeof(uint32_t));
  size_t total = b_acc + b_q + b_p + b_f + b_c;
  if (cap_p > 0xFFFFFFFFull) return fail(RT_ERR_INVALID_ARG, "render grid too large for the drain pools");
  void* base = nullptr;
  cudaError_t e = cudaMalloc(&base, total);
  if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(e, "workspace allocation"); }
  if (ws.base) cudaFree(ws.base);
  char* p = static_cast<char*>(base);
  ws.base = base;
  ws.bytes = total;
  ws.accum = reinterpret_cast<uint32_t*>(p); p += b_acc;
  ws.wq = reinterpret_cast<float4*>(p); p += b_q;
  ws.pool = reinterpret_cast<float4*>(p); p += b_p;
  ws.pool_flag = reinterpret_cast<uint32_t*>(p); p += b_f;
  ws.counters = reinterpret_cast<uint32_t*>(p);
  ws.cap_p = (uint32_t)cap_p;
  ws.epoch = 0;
  // pool flags start below every epoch a render will use
  e = cudaMemset(ws.pool_flag, 0, 2 * cap_p * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();   // before any render stream reads them
  if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(e, "workspace initialisation"); }
  ws.cap_s = cap_s;
  ws.cap_r = cap_r;
  ws.n_warps = n_warps;
  ws.cap_pixels = cap_pixels;
  ws.L = sc->nl;
  return RT_OK;
}

int make_render_args(const rt_scene* scene, const rt_camera* cam, float eye_sep, float convergence,
                     uint32_t W, uint32_t H, uint32_t max_depth, rt::RenderArgs& a) {
  if (!scene) return fail(RT_ERR_INVALID_ARG, "scene is NULL");
  if (!cam) return fail(RT_ERR_INVALID_ARG, "camera is NULL");
  if (W < 1 || H < 1) return fail(RT_ERR_INVALID_ARG, "W and H must be >= 1");
  if (2ull * W * H > (1ull << 31)) return fail(RT_ERR_INVALID_ARG, "2*W*H exceeds 2^31");
  if (max_depth > RT_MAX_DEPTH) return fail(RT_ERR_INVALID_ARG, "max_depth exceeds RT_MAX_DEPTH");
  if (!(std::isfinite(eye_sep) && eye_sep >= 0.f)) return fail(RT_ERR_INVALID_ARG, "eye_sep must be finite and >= 0");
  if (!(std::isfinite(convergence) && convergence > 0.f)) return fail(RT_ERR_INVALID_ARG, "convergence must be finite and > 0");
  if (!finite3(cam->eye) || !finite3(cam->forward) || !finite3(cam->up) ||
      !(cam->vfov_deg > 0.f && cam->vfov_deg < 180.f))
    return fail(RT_ERR_INVALID_ARG, "camera has non-finite values or vfov outside (0,180)");
  const double f[3] = {cam->forward[0], cam->forward[1], cam->forward[2]};
  const double u[3] = {cam->up[0], cam->up[1], cam->up[2]};
  double r[3] = {f[1] * u[2] - f[2] * u[1], f[2] * u[0] - f[0] * u[2], f[0] * u[1] - f[1] * u[0]};
  const double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  const double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  if (!(rl > 0.0) || !(fl > 0.0)) return fail(RT_ERR_INVALID_ARG, "forward x up vanishes");
  double fw[3] = {f[0] / fl, f[1] / fl, f[2] / fl};
  for (double& x : r) x /= rl;
  const double up2[3] = {r[1] * fw[2] - r[2] * fw[1], r[2] * fw[0] - r[0] * fw[2], r[0] * fw[1] - r[1] * fw[0]};
  const double ty = std::tan(0.5 * (double)cam->vfov_deg * M_PI / 180.0);
  std::memset(&a, 0, sizeof a);
  for (int k = 0; k < 3; ++k) {
    a.cam.eye[k] = cam->eye[k];
    a.cam.right[k] = (float)r[k];
    a.cam.up[k] = (float)up2[k];
    a.cam.fwd[k] = (float)fw[k];
  }
  a.cam.tan_y = (float)ty;
  a.cam.tan_x = (float)(ty * (double)W / (double)H);
  a.cam.sx = (float)(2.0 * ty / (double)H);      // 2 tan_x / W = 2 tan_y / H
  a.cam.sy = (float)(2.0 * ty / (double)H);
  a.cam.zc = convergence;
  a.cam.half_sep = 0.5f * eye_sep;
  a.cam.W = W;
  a.cam.H = H;
  a.cam.tiles_x = (W + 7) / 8;
  a.cam.tiles_y = (H + 3) / 4;
  a.cam.y0 = 0;
  a.cam.rows = H;
  // binary renders walk the SAH tree unless the LBVH is asked for; the
  // 4-wide tree (and the work counts of a 4-wide scene) derive from the SAH
  // tree
  a.sc.nodes = scene->tree == RT_TREE_LBVH ? scene->nodes : scene->nodes_sah;
  a.sc.nodes4 = scene->nodes4;
  a.sc.n4 = scene->n4;
  a.sc.n_top = scene->n_top;
  a.tree = scene->tree == RT_TREE_WIDE ? rt::kTreeWide4 : rt::kTreeBinary;
  a.sc.prims = scene->prims;
  a.sc.mats = scene->mats;
  a.sc.lights = scene->lights;
  a.sc.n_prims = scene->n;
  a.sc.n_spheres = scene->ns;
  a.sc.n_mats = scene->nm;
  a.sc.n_lights = scene->nl;
  a.max_depth = max_depth;
  a.color_scale = scene->color_scale;
  a.err = scene->err;
  a.eyes = 3u;
  a.resolve = true;
  a.trace_stage = rt::ST_TRACE;
  return RT_OK;
}

}  // namespace rt

using rt::ensure_workspace;
using rt::make_render_args;

extern "C" {

const char* rt_last_error(void) { return g_last_error.c_str(); }

const char* rt_version(void) { return "rt_stereo 0.1 (sm_103a)"; }

uint32_t rt_scene_num_prims(const rt_scene* scene) { return scene ? scene->n : 0; }

int rt_scene_create(const rt_sphere* spheres, uint32_t n_spheres, const rt_triangle* tris,
                    uint32_t n_tris, const rt_material* mats, uint32_t n_mats,
                    const rt_light* lights, uint32_t n_lights, void* cuda_stream,
                    rt_scene** out_scene) {
  if (!out_scene) return fail(RT_ERR_INVALID_ARG, "out_scene is NULL");
  *out_scene = nullptr;
  const uint64_t n = (uint64_t)n_spheres + n_tris;
  if (n < 1 || n >= (1ull << 31)) return fail(RT_ERR_INVALID_ARG, "need 1 <= n_spheres + n_tris < 2^31");
  if ((n_spheres && !spheres) || (n_tris && !tris)) return fail(RT_ERR_INVALID_ARG, "primitive array is NULL");
  if (n_mats < 1 || !mats) return fail(RT_ERR_INVALID_ARG, "need at least one material");
  if (n_lights < 1 || !lights) return fail(RT_ERR_INVALID_ARG, "need at least one light");
  double bound = 0.5;  // the background's largest channel
  float max_alb = 0.f, sum_i = 0.f;
  for (uint32_t m = 0; m < n_mats; ++m) {
    const rt_material& q = mats[m];
    for (int c = 0; c < 3; ++c) {
      if (!(q.albedo[c] >= 0.f && q.albedo[c] <= 1.f)) return fail(RT_ERR_INVALID_ARG, "albedo outside [0,1] in material " + std::to_string(m));
      max_alb = std::fmax(max_alb, q.albedo[c]);
    }
    if (!(q.reflectivity >= 0.f && q.reflectivity <= 1.f)) return fail(RT_ERR_INVALID_ARG, "reflectivity outside [0,1] in material " + std::to_string(m));
  }
  for (uint32_t l = 0; l < n_lights; ++l) {
    if (!finite3(lights[l].position) || !(lights[l].intensity >= 0.f) || !std::isfinite(lights[l].intensity))
      return fail(RT_ERR_INVALID_ARG, "light " + std::to_string(l) + " invalid");
    sum_i += lights[l].intensity;
  }
  for (uint32_t i = 0; i < n_spheres; ++i) {
    const rt_sphere& s = spheres[i];
    if (!finite3(s.center) || !(s.radius > 0.f) || !std::isfinite(s.radius))
      return fail(RT_ERR_INVALID_ARG, "sphere " + std::to_string(i) + " invalid");
    if (s.material >= n_mats) return fail(RT_ERR_INVALID_ARG, "sphere " + std::to_string(i) + " material out of range");
  }
  for (uint32_t i = 0; i < n_tris; ++i) {
    const rt_triangle& t = tris[i];
    if (!finite3(t.v0) || !finite3(t.v1) || !finite3(t.v2))
      return fail(RT_ERR_INVALID_ARG, "triangle " + std::to_string(i) + " has a non-finite vertex");
    if (t.material >= n_mats) return fail(RT_ERR_INVALID_ARG, "triangle " + std::to_string(i) + " material out of range");
  }
  bound = std::fmax(bound, (double)max_alb * (rt::kAmbient + (double)sum_i));
  if (!std::isfinite(bound) || bound > 1e6) return fail(RT_ERR_INVALID_ARG, "light intensities too large");

  rt_scene* sc = new (std::nothrow) rt_scene();
  if (!sc) return fail(RT_ERR_OOM, "host allocation failed");
  cudaGetDevice(&sc->device);
  sc->ns = n_spheres; sc->nt = n_tris; sc->n = (uint32_t)n; sc->nm = n_mats; sc->nl = n_lights;
  // fixed-point colour scale: the largest power of two with bound * scale <= 2^31
  sc->color_scale = (float)std::ldexp(1.0, (int)std::floor(std::log2(2147483648.0 / bound)));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  const size_t b_nodes = align256((n > 1 ? n - 1 : 1) * 4 * sizeof(float4));
  const size_t b_prims = align256(n * 3 * sizeof(float4));
  const size_t b_mats = align256((size_t)n_mats * sizeof(float4));
  const size_t b_lights = align256((size_t)n_lights * sizeof(float4));
  const size_t b_keys = align256(n * sizeof(uint64_t));
  const size_t b_parent = align256((2 * n - 1) * sizeof(int32_t));
  const size_t b_nodes4 = align256((n > 1 ? n - 1 : 1) * 7 * sizeof(float4));
  const size_t b_err = 256;
  const size_t total = 2 * b_nodes + b_prims + b_mats + b_lights + b_keys + b_parent + b_nodes4 + b_err;
  cudaError_t e = cudaMalloc(&sc->block, total);
  if (e != cudaSuccess) { cudaGetLastError(); delete sc; return cuda_fail(e, "scene allocation"); }
  char* p = static_cast<char*>(sc->block);
  sc->nodes = reinterpret_cast<float4*>(p); p += b_nodes;
  sc->prims = reinterpret_cast<float4*>(p); p += b_prims;
  sc->mats = reinterpret_cast<float4*>(p); p += b_mats;
  sc->lights = reinterpret_cast<float4*>(p); p += b_lights;
  sc->keys = reinterpret_cast<uint64_t*>(p); p += b_keys;
  sc->parent = reinterpret_cast<int32_t*>(p); p += b_parent;
  sc->nodes4 = reinterpret_cast<float4*>(p); p += b_nodes4;
  sc->nodes_sah = reinterpret_cast<float4*>(p); p += b_nodes;
  sc->err = reinterpret_cast<uint32_t*>(p);
  e = cudaMallocHost(&sc->h_err, sizeof(uint32_t));
  if (e != cudaSuccess) { cudaGetLastError(); cudaFree(sc->block); delete sc; return cuda_fail(e, "pinned allocation"); }
  *sc->h_err = 0;

  // temporary: raw input records + LBVH scratch
  const size_t b_sph = align256((size_t)n_spheres * sizeof(rt_sphere) + 16);
  const size_t b_tri = align256((size_t)n_tris * sizeof(rt_triangle) + 16);
  const size_t b_tmp = align256(std::max(rt::lbvh_tmp_bytes((uint32_t)n), rt::sah_tmp_bytes((uint32_t)n)));
  void* tmp = nullptr;
  e = cudaMalloc(&tmp, b_sph + b_tri + b_tmp + 256);
  if (e != cudaSuccess) { cudaGetLastError(); rt_scene_destroy(sc); return cuda_fail(e, "build scratch allocation"); }
  char* tp = static_cast<char*>(tmp);
  float4* d_sph = reinterpret_cast<float4*>(tp);
  float* d_tri = reinterpret_cast<float*>(tp + b_sph);
  void* d_lbvh = tp + b_sph + b_tri;
  if (n_spheres) cudaMemcpyAsync(d_sph, spheres, (size_t)n_spheres * sizeof(rt_sphere), cudaMemcpyHostToDevice, st);
  if (n_tris) cudaMemcpyAsync(d_tri, tris, (size_t)n_tris * sizeof(rt_triangle), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(sc->mats, mats, (size_t)n_mats * sizeof(float4), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(sc->lights, lights, (size_t)n_lights * sizeof(float4), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(sc->err, 0, sizeof(uint32_t), st);
  e = rt::build_lbvh(d_sph, d_tri, n_spheres, n_tris, sc->nodes, sc->prims, sc->keys, sc->parent,
                     d_lbvh, b_tmp, sc->err, st);
  // the render tree: SAH splits over the LBVH's leaves
  if (e == cudaSuccess)
    e = rt::build_sah_tree(sc->nodes, sc->parent, (uint32_t)n, sc->nodes_sah, d_lbvh, sc->err, st);
  // (the 4-wide tree is built when a render first asks for it:
  // rt_scene_set_traversal)
  if (e == cudaSuccess) e = cudaMemcpyAsync(sc->h_err, sc->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(tmp);
  if (e != cudaSuccess) { rt_scene_destroy(sc); return cuda_fail(e, "BVH build"); }
  if (*sc->h_err) {
    uint32_t bits = *sc->h_err;
    rt_scene_destroy(sc);
    return fail(RT_ERR_DEVICE_CHECK, "BVH build device check failed (bits " + std::to_string(bits) + ")");
  }
  *out_scene = sc;
  return RT_OK;
}

void rt_scene_destroy(rt_scene* scene) {
  if (!scene) return;
  free_workspace(scene->ws);
  if (scene->block) cudaFree(scene->block);
  if (scene->h_err) cudaFreeHost(scene->h_err);
  delete scene;
}

int rt_render_stereo_aux(const rt_scene* scene, const rt_camera* cam, float eye_sep,
                         float convergence, uint32_t W, uint32_t H, uint32_t max_depth,
                         float* out_L, float* out_R, uint32_t* hit_id_L, uint32_t* hit_id_R,
                         float* depth_L, float* depth_R, uint64_t* ray_counts, uint64_t* work,
                         void* cuda_stream) {
  rt::RenderArgs a;
  int rc = make_render_args(scene, cam, eye_sep, convergence, W, H, max_depth, a);
  if (rc) return rc;
  if (!out_L || !out_R) return fail(RT_ERR_INVALID_ARG, "output buffer is NULL");
  rc = ensure_workspace(scene, W, H);
  if (rc) return rc;
  a.out_L = out_L; a.out_R = out_R;
  a.hit_L = hit_id_L; a.hit_R = hit_id_R;
  a.depth_L = depth_L; a.depth_R = depth_R;
  a.ray_counts = ray_counts;
  a.work = work;
  if (work) a.tree = rt::kTreeBinary;   // the instrumented walk is binary
  rt::Workspace& ws = const_cast<rt_scene*>(scene)->ws;
  rt::profile_begin(ws, static_cast<cudaStream_t>(cuda_stream));
  cudaError_t e = rt::render(a, ws, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(e, "render launch");
  return RT_OK;
}

int rt_render_stereo(const rt_scene* scene, const rt_camera* cam, float eye_sep, float convergence,
                     uint32_t W, uint32_t H, uint32_t max_depth, float* out_L, float* out_R,
                     void* cuda_stream) {
  return rt_render_stereo_aux(scene, cam, eye_sep, convergence, W, H, max_depth, out_L, out_R,
                              nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, cuda_stream);
}

int rt_render_stereo_rows(const rt_scene* scene, const rt_camera* cam, float eye_sep,
                          float convergence, uint32_t W, uint32_t H, uint32_t max_depth,
                          uint32_t row0, uint32_t n_rows, float* out_L, float* out_R,
                          uint64_t* ray_counts, void* cuda_stream) {
  rt::RenderArgs a;
  int rc = make_render_args(scene, cam, eye_sep, convergence, W, H, max_depth, a);
  if (rc) return rc;
  if (n_rows < 1 || row0 >= H || n_rows > H - row0)
    return fail(RT_ERR_INVALID_ARG, "rows row0 .. row0 + n_rows - 1 must lie inside 0 .. H - 1");
  if (!out_L || !out_R) return fail(RT_ERR_INVALID_ARG, "output buffer is NULL");
  rc = ensure_workspace(scene, W, n_rows);
  if (rc) return rc;
  a.cam.y0 = row0;
  a.cam.rows = n_rows;
  a.cam.tiles_y = (n_rows + 3) / 4;
  a.out_L = out_L; a.out_R = out_R;
  a.ray_counts = ray_counts;
  rt::Workspace& ws = const_cast<rt_scene*>(scene)->ws;
  rt::profile_begin(ws, static_cast<cudaStream_t>(cuda_stream));
  cudaError_t e = rt::render(a, ws, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(e, "row-band render launch");
  return RT_OK;
}

namespace {
// device address of a host buffer the GPU can write directly (pinned and
// mapped; on GB300 the write goes over the coherent CPU-GPU link), or null
float* device_view(float* host) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, host) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
  return static_cast<float*>(at.devicePointer);
}
}  // namespace

int rt_render_stereo_host(const rt_scene* scene, const rt_camera* cam, float eye_sep,
                          float convergence, uint32_t W, uint32_t H, uint32_t max_depth,
                          float* host_L, float* host_R, void* cuda_stream) {
  if (!host_L || !host_R) return fail(RT_ERR_INVALID_ARG, "host output buffer is NULL");
  if (!scene) return fail(RT_ERR_INVALID_ARG, "scene is NULL");
  rt_scene* sc = const_cast<rt_scene*>(scene);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // pinned, device-mapped host buffers: the resolve kernel writes them directly
  float* vL = device_view(host_L);
  float* vR = vL ? device_view(host_R) : nullptr;
  if (vL && vR) {
    int rc = rt_render_stereo(scene, cam, eye_sep, convergence, W, H, max_depth, vL, vR, cuda_stream);
    if (rc) return rc;
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "render to host memory");
    return RT_OK;
  }
  // otherwise render to scene-owned device frames and copy
  const size_t bytes = 2ull * W * H * 3 * sizeof(float);
  if (2ull * W * H <= (1ull << 31) && sc->ws.frame_bytes < bytes) {
    if (sc->ws.frame) cudaFree(sc->ws.frame);
    sc->ws.frame = nullptr;
    sc->ws.frame_bytes = 0;
    cudaError_t e = cudaMalloc(&sc->ws.frame, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(e, "frame allocation"); }
    sc->ws.frame_bytes = bytes;
  }
  float* dL = reinterpret_cast<float*>(sc->ws.frame);
  float* dR = dL + (size_t)W * H * 3;
  int rc = rt_render_stereo(scene, cam, eye_sep, convergence, W, H, max_depth, dL, dR, cuda_stream);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(host_L, dL, bytes / 2, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_R, dR, bytes / 2, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
  return RT_OK;
}

int rt_render_stereo_sequence(const rt_scene* scene, const rt_camera* cams, uint32_t n_frames,
                              float eye_sep, float convergence, uint32_t W, uint32_t H,
                              uint32_t max_depth, float* const* host_L, float* const* host_R,
                              void* cuda_stream) {
  if (!scene) return fail(RT_ERR_INVALID_ARG, "scene is NULL");
  if (n_frames == 0) return RT_OK;
  if (!cams || !host_L || !host_R) return fail(RT_ERR_INVALID_ARG, "camera or host pointer array is NULL");
  for (uint32_t f = 0; f < n_frames; ++f)
    if (!host_L[f] || !host_R[f]) return fail(RT_ERR_INVALID_ARG, "host output buffer of frame " + std::to_string(f) + " is NULL");
  rt::RenderArgs a;
  for (uint32_t f = 0; f < n_frames; ++f) {        // validate every camera before any work
    const int rc = make_render_args(scene, &cams[f], eye_sep, convergence, W, H, max_depth, a);
    if (rc) return rc;
  }
  int rc = ensure_workspace(scene, W, H);
  if (rc) return rc;
  rt_scene* sc = const_cast<rt_scene*>(scene);
  rt::Workspace& ws = sc->ws;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t img = (size_t)W * H * 3;            // floats per image
  const size_t slot = 2 * img * sizeof(float);     // both images
  cudaError_t e = cudaSuccess;
  if (!ws.seq_copy) {
    e = cudaStreamCreateWithFlags(&ws.seq_copy, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&ws.seq_rendered[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ws.seq_copied[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(e, "sequence stream and events"); }
  }
  if (ws.seq_frame_bytes < slot) {
    cudaStreamSynchronize(ws.seq_copy);            // no copy may still read the old slots
    if (ws.seq_frame) cudaFree(ws.seq_frame);
    ws.seq_frame = nullptr;
    ws.seq_frame_bytes = 0;
    e = cudaMalloc(&ws.seq_frame, 2 * slot);
    if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(e, "sequence frame allocation"); }
    ws.seq_frame_bytes = slot;
  }
  for (uint32_t f = 0; f < n_frames && e == cudaSuccess; ++f) {
    const int k = (int)(f & 1u);
    float* dL = ws.seq_frame + (size_t)k * 2 * img;
    float* dR = dL + img;
    // the slot's previous copy (frame f - 2) has to finish before it is overwritten
    if (f >= 2) e = cudaStreamWaitEvent(st, ws.seq_copied[k], 0);
    if (e != cudaSuccess) break;
    rc = make_render_args(scene, &cams[f], eye_sep, convergence, W, H, max_depth, a);
    if (rc) { cudaStreamSynchronize(ws.seq_copy); return rc; }
    a.out_L = dL;
    a.out_R = dR;
    rt::profile_begin(ws, st);
    e = rt::render(a, ws, st);
    if (e == cudaSuccess) e = cudaEventRecord(ws.seq_rendered[k], st);
    // the copy engine reads the finished pair while the next frame renders
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ws.seq_copy, ws.seq_rendered[k], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_L[f], dL, img * sizeof(float), cudaMemcpyDeviceToHost, ws.seq_copy);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_R[f], dR, img * sizeof(float), cudaMemcpyDeviceToHost, ws.seq_copy);
    if (e == cudaSuccess) e = cudaEventRecord(ws.seq_copied[k], ws.seq_copy);
  }
  const cudaError_t e2 = cudaStreamSynchronize(ws.seq_copy);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(e, "sequence render"); }
  return RT_OK;
}

int rt_sync_status(const rt_scene* scene, void* cuda_stream) {
  if (!scene) return fail(RT_ERR_INVALID_ARG, "scene is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaMemcpyAsync(scene->h_err, scene->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  const uint32_t bits = *scene->h_err;
  if (!bits) return RT_OK;
  cudaMemsetAsync(scene->err, 0, sizeof(uint32_t), st);
  cudaStreamSynchronize(st);
  if (bits & rt::ERR_ITER) return fail(RT_ERR_TIMEOUT, "a device loop reached its iteration bound (bits " + std::to_string(bits) + ")");
  return fail(RT_ERR_DEVICE_CHECK, "device-side check failed (bits " + std::to_string(bits) + ")");
}

int rt_scene_get_bvh(const rt_scene* scene, uint64_t* keys, int32_t* left, int32_t* right,
                     int32_t* parent, float* inner_box, float* leaf_box) {
  if (!scene) return fail(RT_ERR_INVALID_ARG, "scene is NULL");
  const uint32_t n = scene->n;
  std::vector<float4> nodes((size_t)(n > 1 ? n - 1 : 0) * 4);
  std::vector<int32_t> par(2 * (size_t)n - 1);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && keys) e = cudaMemcpy(keys, scene->keys, (size_t)n * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && !nodes.empty()) e = cudaMemcpy(nodes.data(), scene->nodes, nodes.size() * sizeof(float4), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(par.data(), scene->parent, par.size() * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "BVH download");
  if (parent) std::memcpy(parent, par.data(), par.size() * 4);
  auto child_box = [&](uint32_t p, int slot, float* out) {
    const float* f = reinterpret_cast<const float*>(&nodes[4 * (size_t)p]);
    if (slot == 0) { out[0] = f[0]; out[3] = f[1]; out[1] = f[2]; out[4] = f[3]; out[2] = f[8]; out[5] = f[9]; }
    else { out[0] = f[4]; out[3] = f[5]; out[1] = f[6]; out[4] = f[7]; out[2] = f[10]; out[5] = f[11]; }
  };
  for (uint32_t i = 0; i + 1 < n; ++i) {
    const float4 c = nodes[4 * (size_t)i + 3];
    const int32_t l = __builtin_bit_cast(int32_t, c.x), r = __builtin_bit_cast(int32_t, c.y);
    if (left) left[i] = l;
    if (right) right[i] = r;
    if (leaf_box) {
      if (l < 0) child_box(i, 0, leaf_box + 6 * (size_t)~l);
      if (r < 0) child_box(i, 1, leaf_box + 6 * (size_t)~r);
    }
    if (inner_box) {
      if (l >= 0) child_box(i, 0, inner_box + 6 * (size_t)l);
      if (r >= 0) child_box(i, 1, inner_box + 6 * (size_t)r);
    }
  }
  if (inner_box && n > 1) {  // the root's box is the union of its children
    float b0[6], b1[6];
    child_box(0, 0, b0);
    child_box(0, 1, b1);
    for (int k = 0; k < 3; ++k) { inner_box[k] = std::fmin(b0[k], b1[k]); inner_box[3 + k] = std::fmax(b0[3 + k], b1[3 + k]); }
  }
  if (leaf_box && n == 1) {  // single primitive: its box sits in the spare node slot
    std::vector<float4> spare(4);
    e = cudaMemcpy(spare.data(), scene->nodes, 4 * sizeof(float4), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "BVH download");
    nodes.swap(spare);
    child_box(0, 0, leaf_box);
  }
  return RT_OK;
}

int rt_debug_set_node(rt_scene* scene, uint32_t node, int32_t left, int32_t right,
                      int empty_right) {
  if (!scene) return fail(RT_ERR_INVALID_ARG, "scene is NULL");
  const int64_t n = scene->n;
  auto ok = [&](int32_t c) { return c >= 0 ? (int64_t)c < n - 1 : (int64_t)~c < n; };
  if ((int64_t)node >= n - 1 || !ok(left) || !ok(right))
    return fail(RT_ERR_INVALID_ARG, "node or child index out of range");
  float4 nd[4];
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(nd, scene->nodes + 4 * (size_t)node, sizeof nd, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "node download");
  nd[3].x = __builtin_bit_cast(float, left);
  nd[3].y = __builtin_bit_cast(float, right);
  if (empty_right) {  // lo > hi on every axis
    nd[1] = make_float4(1.f, -1.f, 1.f, -1.f);
    nd[2].z = 1.f;
    nd[2].w = -1.f;
  }
  e = cudaMemcpy(scene->nodes + 4 * (size_t)node, nd, sizeof nd, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "node upload");
  return RT_OK;
}

int rt_debug_get_sah_tree(const rt_scene* scene, float* nodes) {
  if (!scene || !nodes) return fail(RT_ERR_INVALID_ARG, "scene or nodes is NULL");
  if (scene->n < 2) return RT_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(nodes, scene->nodes_sah, (size_t)(scene->n - 1) * 4 * sizeof(float4),
                   cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "SAH tree download");
  return RT_OK;
}

int rt_debug_set_sah_slicing(int enable) {
  rt::set_sah_slicing(enable != 0);
  return RT_OK;
}

int rt_debug_set_pool_capacity(rt_scene* scene, uint32_t entries) {
  if (!scene) return fail(RT_ERR_INVALID_ARG, "scene is NULL");
  scene->ws.cap_p_limit = entries;
  return RT_OK;
}

int rt_scene_set_traversal(rt_scene* scene, int tree) {
  if (!scene) return fail(RT_ERR_INVALID_ARG, "scene is NULL");
  if (tree != RT_TREE_SAH && tree != RT_TREE_WIDE && tree != RT_TREE_LBVH)
    return fail(RT_ERR_INVALID_ARG, "tree must be RT_TREE_SAH, RT_TREE_WIDE or RT_TREE_LBVH");
  if (tree == RT_TREE_WIDE && !scene->wide_built && scene->n > 1) {
    // the 4-wide tree, collapsed from the SAH tree (1.28 against 1.40 ms on
    // the 1080p blob pair when collapsed from the LBVH); scratch: the build's
    // own, then the SAH tree's inner parents, then two counts
    const uint32_t n = scene->n;
    const size_t b4 = align256(rt::bvh4_tmp_bytes(n)), bp = align256(4 * (size_t)n);
    void* tmp = nullptr;
    cudaError_t e = cudaSetDevice(scene->device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMalloc(&tmp, b4 + bp + 256);
    if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(e, "4-wide tree scratch"); }
    char* t = static_cast<char*>(tmp);
    int32_t* sah_parent = reinterpret_cast<int32_t*>(t + b4);
    uint32_t* d_counts = reinterpret_cast<uint32_t*>(t + b4 + bp);
    uint32_t counts[2] = {0, 0};
    e = cudaMemset(d_counts, 0, 2 * sizeof(uint32_t));
    if (e == cudaSuccess) e = rt::inner_parents(scene->nodes_sah, n, sah_parent, 0);
    if (e == cudaSuccess)
      e = rt::build_bvh4(scene->nodes_sah, sah_parent, n, rt::treelet_depth(), scene->nodes4, d_counts,
                         tmp, 0);
    if (e == cudaSuccess) e = cudaMemcpy(counts, d_counts, sizeof counts, cudaMemcpyDeviceToHost);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(e, "4-wide tree build");
    scene->n_top = counts[0];
    scene->n4 = counts[1];
    scene->wide_built = true;
  }
  scene->tree = tree;
  return RT_OK;
}

int rt_profile_enable(rt_scene* scene, int on) {
  if (!scene) return fail(RT_ERR_INVALID_ARG, "scene is NULL");
  rt::Workspace& ws = scene->ws;
  if (on && !ws.ev[0]) {
    for (cudaEvent_t& e : ws.ev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return cuda_fail(r, "event creation");
    }
  }
  ws.profile = on != 0;
  ws.n_ev = 0;
  return RT_OK;
}

int rt_profile_read(const rt_scene* scene, float* ms) {
  if (!scene || !ms) return fail(RT_ERR_INVALID_ARG, "scene or ms is NULL");
  const rt::Workspace& ws = scene->ws;
  if (!ws.profile || ws.n_ev < 2) return fail(RT_ERR_INVALID_ARG, "no profiled render");
  cudaError_t e = cudaEventSynchronize(ws.ev[ws.n_ev - 1]);
  if (e != cudaSuccess) return cuda_fail(e, "event wait");
  for (int k = 0; k < rt::ST_COUNT; ++k) ms[k] = 0.f;
  for (int k = 1; k < ws.n_ev; ++k) {
    float t = 0.f;
    e = cudaEventElapsedTime(&t, ws.ev[k - 1], ws.ev[k]);
    if (e != cudaSuccess) return cuda_fail(e, "event time");
    ms[ws.ev_stage[k]] += t;
  }
  return RT_OK;
}

}  // extern "C"
