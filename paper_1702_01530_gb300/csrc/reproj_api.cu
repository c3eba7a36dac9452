// C-ABI of the learned right-eye reprojection and its retrace network
// (declared in include/rt_stereo.h). Host-side marshalling and buffer
// ownership only; the work runs in reproj.cu, nn.cu and trace.cu.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include <algorithm>

#include "rt_internal.cuh"

using rt::cuda_fail;
using rt::fail;

struct rt_net {
  void* block = nullptr;        // params, grads, Adam m and v, packed weights, scalars
  float* params = nullptr;
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* wf[4] = {};
  __nv_bfloat16* wb[4] = {};
  float* loss = nullptr;
  uint32_t* err = nullptr;
  uint32_t step = 0;
  // forward / training activations, grown on demand
  void* tb = nullptr;
  uint64_t tcap = 0;
  __nv_bfloat16* act[3] = {};
  float* prob = nullptr;
  __nv_bfloat16* g16 = nullptr;
  float* g32 = nullptr;
  __nv_bfloat16* dz[2] = {};
  float* wpart = nullptr;       // per-CTA partial sums of the weight gradients
  // FP8 inference (rt_net_set_fp8): E4M3 weights of layers 2-4, their
  // per-output-channel scales and the inverse scales the epilogues apply
  bool fp8 = false;
  float act_scale[3] = {1.f, 1.f, 1.f};
  uint8_t* w8[3] = {};
  float* wscale[3] = {};
  float* inv[3] = {};
  unsigned* amax = nullptr;
};

namespace {

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

// the network's forward pass in the precision it is set to (BF16, or FP8
// after rt_net_set_fp8); act: three scratch maps of W*H*32 BF16 each
cudaError_t net_forward(rt_net* net, const __nv_bfloat16* feat16, __nv_bfloat16* const act[3],
                        float* prob, uint32_t W, uint32_t H, cudaStream_t st, uint32_t n_img = 1) {
  if (!net->fp8)
    return rt::nn::forward(feat16, net->params, net->wf, act[0], act[1], act[2], prob, W, H, net->err, st,
                           n_img);
  return rt::nn::forward_fp8(feat16, net->params, net->wf, net->w8, net->inv, net->act_scale,
                             reinterpret_cast<uint8_t*>(act[0]), reinterpret_cast<uint8_t*>(act[1]),
                             reinterpret_cast<uint8_t*>(act[2]), prob, W, H, net->err, st, n_img);
}

int net_buffers(rt_net* net, uint64_t P) {
  if (net->tb && net->tcap >= P) return RT_OK;
  const size_t b_act = a256(P * 32 * 2), b_prob = a256(P * 4), b_g16 = a256(P * 16 * 2),
               b_g32 = a256(P * 4), b_part = a256(rt::nn::wgrad_part_floats(0xFFFFFFFFu) * 4);
  void* base = nullptr;
  cudaError_t e = cudaMalloc(&base, 3 * b_act + b_prob + b_g16 + b_g32 + 2 * b_act + b_part);
  if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(e, "network activations"); }
  if (net->tb) cudaFree(net->tb);
  net->tb = base;
  net->tcap = P;
  char* p = static_cast<char*>(base);
  for (int i = 0; i < 3; ++i) { net->act[i] = reinterpret_cast<__nv_bfloat16*>(p); p += b_act; }
  net->prob = reinterpret_cast<float*>(p); p += b_prob;
  net->g16 = reinterpret_cast<__nv_bfloat16*>(p); p += b_g16;
  net->g32 = reinterpret_cast<float*>(p); p += b_g32;
  for (int i = 0; i < 2; ++i) { net->dz[i] = reinterpret_cast<__nv_bfloat16*>(p); p += b_act; }
  net->wpart = reinterpret_cast<float*>(p);
  return RT_OK;
}

int reproj_buffers(const rt_scene* sc_c, uint64_t P) {
  rt_scene* sc = const_cast<rt_scene*>(sc_c);
  rt::ReprojBuffers& rp = sc->ws.rp;
  if (rp.base && rp.cap >= P) return RT_OK;
  const size_t b4 = a256(P * 4), b12 = a256(P * 12), b8 = a256(P * 8), b1 = a256(P),
               bf = a256(P * 16 * 2), bact = a256(P * 32 * 2);
  const size_t total = b4 + b12 + b4 + b4 + b8 + bf + b1 + b12 + b1 + b4 + 256 + b4 + 3 * bact;
  void* base = nullptr;
  cudaError_t e = cudaMalloc(&base, total);
  if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(e, "reprojection buffers"); }
  if (rp.base) cudaFree(rp.base);
  char* p = static_cast<char*>(base);
  rp.base = base;
  rp.cap = P;
  rp.depth_L = reinterpret_cast<float*>(p); p += b4;
  rp.normal_L = reinterpret_cast<float*>(p); p += b12;
  rp.refl_L = reinterpret_cast<float*>(p); p += b4;
  rp.id_L = reinterpret_cast<uint32_t*>(p); p += b4;
  rp.zbuf = reinterpret_cast<unsigned long long*>(p); p += b8;
  rp.feat16 = reinterpret_cast<__nv_bfloat16*>(p); p += bf;
  rp.hole = reinterpret_cast<uint8_t*>(p); p += b1;
  rp.warped = reinterpret_cast<float*>(p); p += b12;
  rp.mask = reinterpret_cast<uint8_t*>(p); p += b1;
  rp.plist = reinterpret_cast<uint32_t*>(p); p += b4;
  rp.count = reinterpret_cast<uint32_t*>(p); p += 256;
  rp.prob = reinterpret_cast<float*>(p); p += b4;
  for (int i = 0; i < 3; ++i) { rp.act[i] = reinterpret_cast<__nv_bfloat16*>(p); p += bact; }
  return RT_OK;
}

// CRC-32 of the IEEE 802.3 / zlib convention (reflected polynomial
// 0xEDB88320, initial value and final xor 0xFFFFFFFF), bit by bit
uint32_t crc32(const unsigned char* p, size_t n) {
  uint32_t c = 0xFFFFFFFFu;
  for (size_t i = 0; i < n; ++i) {
    c ^= p[i];
    for (int k = 0; k < 8; ++k) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
  }
  return c ^ 0xFFFFFFFFu;
}

// Training checkpoint: everything needed to continue training exactly where
// it stopped. Little-endian, no padding:
//   char magic[8] = "RTNETCK1"; uint32 version (1), n_params, adam_step,
//   fp8 (0/1); float act_scale[3]; float params[n], adam_m[n], adam_v[n];
//   uint32 CRC-32 of every byte before it.
constexpr char kCkptMagic[8] = {'R', 'T', 'N', 'E', 'T', 'C', 'K', '1'};
constexpr uint32_t kCkptVersion = 1;
constexpr size_t kCkptHeader = 8 + 4 * 4 + 3 * 4;

// largest power of two s with amax * s <= 448 (the E4M3 maximum), 1 for
// amax = 0, kept within the [2^-30, 2^30] that rt_net_set_fp8 accepts
float fp8_pow2_scale(float amax) {
  if (!(amax > 0.f)) return 1.f;
  int k = 0;
  std::frexp(448.0 / (double)amax, &k);        // 448 / amax = m 2^k, m in [0.5, 1)
  double s = std::ldexp(1.0, k - 1);
  while ((double)amax * s > 448.0) s *= 0.5;   // a rounded quotient could reach 2^k
  return (float)std::min(std::max(s, std::ldexp(1.0, -30)), std::ldexp(1.0, 30));
}

float focal_px(const rt_camera* cam, uint32_t H) {
  return (float)(0.5 * (double)H / std::tan(0.5 * (double)cam->vfov_deg * M_PI / 180.0));
}

}  // namespace

extern "C" {

int rt_net_create(const float* host_params, uint32_t n_params, rt_net** out) {
  if (!out) return fail(RT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!host_params || n_params != rt::nn::kParams)
    return fail(RT_ERR_INVALID_ARG, "need RT_NET_PARAMS (" + std::to_string(rt::nn::kParams) + ") parameters");
  for (uint32_t i = 0; i < n_params; ++i)
    if (!std::isfinite(host_params[i])) return fail(RT_ERR_INVALID_ARG, "non-finite parameter " + std::to_string(i));
  rt_net* net = new (std::nothrow) rt_net();
  if (!net) return fail(RT_ERR_OOM, "host allocation failed");
  const size_t bp = a256((size_t)rt::nn::kParams * 4);
  size_t bw = 0;
  for (int l = 0; l < 4; ++l) bw += a256(rt::nn::packed_fwd_elems(l) * 2) + a256(rt::nn::packed_bwd_elems(l) * 2);
  size_t b8 = 256;                                          // amax
  for (int l = 1; l < 4; ++l) b8 += a256(rt::nn::packed_fp8_bytes(l)) + 2 * 256;
  cudaError_t e = cudaMalloc(&net->block, 4 * bp + bw + 512 + b8);
  if (e != cudaSuccess) { cudaGetLastError(); delete net; return cuda_fail(e, "network allocation"); }
  char* p = static_cast<char*>(net->block);
  net->params = reinterpret_cast<float*>(p); p += bp;
  net->grads = reinterpret_cast<float*>(p); p += bp;
  net->m = reinterpret_cast<float*>(p); p += bp;
  net->v = reinterpret_cast<float*>(p); p += bp;
  for (int l = 0; l < 4; ++l) {
    net->wf[l] = reinterpret_cast<__nv_bfloat16*>(p); p += a256(rt::nn::packed_fwd_elems(l) * 2);
    net->wb[l] = reinterpret_cast<__nv_bfloat16*>(p); p += a256(rt::nn::packed_bwd_elems(l) * 2);
  }
  net->loss = reinterpret_cast<float*>(p); p += 256;
  net->err = reinterpret_cast<uint32_t*>(p); p += 256;
  for (int l = 1; l < 4; ++l) {
    net->w8[l - 1] = reinterpret_cast<uint8_t*>(p); p += a256(rt::nn::packed_fp8_bytes(l));
    net->wscale[l - 1] = reinterpret_cast<float*>(p); p += 256;
    net->inv[l - 1] = reinterpret_cast<float*>(p); p += 256;
  }
  net->amax = reinterpret_cast<unsigned*>(p);
  e = cudaMemcpy(net->params, host_params, (size_t)n_params * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(net->m, 0, (size_t)n_params * 4);
  if (e == cudaSuccess) e = cudaMemset(net->v, 0, (size_t)n_params * 4);
  if (e == cudaSuccess) e = cudaMemset(net->err, 0, 4);
  if (e == cudaSuccess) e = rt::nn::pack_weights(net->params, net->wf, net->wb, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { cudaFree(net->block); delete net; return cuda_fail(e, "network upload"); }
  *out = net;
  return RT_OK;
}

void rt_net_destroy(rt_net* net) {
  if (!net) return;
  if (net->tb) cudaFree(net->tb);
  if (net->block) cudaFree(net->block);
  delete net;
}

int rt_net_get_params(const rt_net* net, float* host_params) {
  if (!net || !host_params) return fail(RT_ERR_INVALID_ARG, "net or output is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(host_params, net->params, (size_t)rt::nn::kParams * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "parameter download");
  return RT_OK;
}

int rt_net_status(const rt_net* net, void* cuda_stream) {
  if (!net) return fail(RT_ERR_INVALID_ARG, "net is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  uint32_t bits = 0;
  cudaError_t e = cudaMemcpyAsync(&bits, net->err, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (!bits) return RT_OK;
  cudaMemsetAsync(net->err, 0, 4, st);
  cudaStreamSynchronize(st);
  return fail(RT_ERR_TIMEOUT, "a tensor-core wait reached its bound (bits " + std::to_string(bits) + ")");
}

int rt_net_set_fp8(rt_net* net, const float* act_scales) {
  if (!net) return fail(RT_ERR_INVALID_ARG, "net is NULL");
  if (!act_scales) { net->fp8 = false; return RT_OK; }
  for (int i = 0; i < 3; ++i) {
    int k = 0;
    const double m = std::frexp((double)act_scales[i], &k);
    if (!(act_scales[i] > 0.f) || !std::isfinite(act_scales[i]) || m != 0.5 || k < -29 || k > 31)
      return fail(RT_ERR_INVALID_ARG, "activation scales must be powers of two in [2^-30, 2^30]");
  }
  std::vector<float> h(rt::nn::kParams);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), net->params, h.size() * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "rt_net_set_fp8: parameter download");
  // per output channel of layers 2-4: the largest power of two s with
  // max |w| * s <= 448 (1 for an all-zero channel); inverse scale 1/(a s)
  static const uint32_t off_w[4] = {0, 2912, 12160, 21408};
  static const int cout[4] = {32, 32, 32, 1}, cin[4] = {10, 32, 32, 32};
  for (int l = 1; l < 4; ++l) {
    float sc[32], iv[32];
    for (int co = 0; co < 32; ++co) {
      double amax = 0.0;
      if (co < cout[l])
        for (int j = 0; j < cin[l] * 9; ++j)
          amax = std::max(amax, (double)std::fabs(h[off_w[l] + (size_t)co * cin[l] * 9 + j]));
      double s = 1.0;
      if (amax > 0.0) {
        int k = 0;
        std::frexp(448.0 / amax, &k);
        s = std::ldexp(1.0, k - 1);
      }
      sc[co] = (float)s;
      iv[co] = (float)(1.0 / ((double)act_scales[l - 1] * s));
    }
    e = cudaMemcpy(net->wscale[l - 1], sc, sizeof sc, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(net->inv[l - 1], iv, sizeof iv, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "rt_net_set_fp8: scale upload");
  }
  e = rt::nn::pack_weights_fp8(net->params, net->wscale, net->w8, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "rt_net_set_fp8: weight packing");
  for (int i = 0; i < 3; ++i) net->act_scale[i] = act_scales[i];
  net->fp8 = true;
  return RT_OK;
}

int rt_net_activation_amax(rt_net* net, const uint16_t* d_feat16, uint32_t W, uint32_t H,
                           float* host_amax, void* cuda_stream) {
  if (!net || !d_feat16 || !host_amax || W < 1 || H < 1) return fail(RT_ERR_INVALID_ARG, "bad argument");
  if ((uint64_t)W * H > (1ull << 30)) return fail(RT_ERR_INVALID_ARG, "image too large");
  int rc = net_buffers(net, (uint64_t)W * H);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaMemsetAsync(net->amax, 0, 3 * sizeof(unsigned), st);
  if (e == cudaSuccess)
    e = rt::nn::forward(reinterpret_cast<const __nv_bfloat16*>(d_feat16), net->params, net->wf,
                        net->act[0], net->act[1], net->act[2], net->prob, W, H, net->err, st);
  if (e == cudaSuccess) e = rt::nn::activation_amax(net->act, (uint64_t)W * H, net->amax, st);
  unsigned bits[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(bits, net->amax, sizeof bits, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "rt_net_activation_amax");
  for (int i = 0; i < 3; ++i) std::memcpy(&host_amax[i], &bits[i], 4);
  return RT_OK;
}

int rt_net_calibrate_fp8(rt_net* net, const uint16_t* const* d_feats, uint32_t n_maps, uint32_t W,
                         uint32_t H, float* host_amax, float* host_scales, void* cuda_stream) {
  if (!net || !d_feats || n_maps < 1 || W < 1 || H < 1) return fail(RT_ERR_INVALID_ARG, "bad argument");
  if ((uint64_t)W * H > (1ull << 30)) return fail(RT_ERR_INVALID_ARG, "image too large");
  for (uint32_t i = 0; i < n_maps; ++i)
    if (!d_feats[i]) return fail(RT_ERR_INVALID_ARG, "feature map " + std::to_string(i) + " is NULL");
  int rc = net_buffers(net, (uint64_t)W * H);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // maxima of the BF16 network's three hidden activations over every map
  cudaError_t e = cudaMemsetAsync(net->amax, 0, 3 * sizeof(unsigned), st);
  for (uint32_t i = 0; i < n_maps && e == cudaSuccess; ++i) {
    e = rt::nn::forward(reinterpret_cast<const __nv_bfloat16*>(d_feats[i]), net->params, net->wf,
                        net->act[0], net->act[1], net->act[2], net->prob, W, H, net->err, st);
    if (e == cudaSuccess) e = rt::nn::activation_amax(net->act, (uint64_t)W * H, net->amax, st);
  }
  unsigned bits[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(bits, net->amax, sizeof bits, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "rt_net_calibrate_fp8");
  float amax[3], scales[3];
  for (int i = 0; i < 3; ++i) {
    std::memcpy(&amax[i], &bits[i], 4);
    scales[i] = fp8_pow2_scale(amax[i]);
  }
  rc = rt_net_set_fp8(net, scales);
  if (rc) return rc;
  for (int i = 0; i < 3; ++i) {
    if (host_amax) host_amax[i] = amax[i];
    if (host_scales) host_scales[i] = scales[i];
  }
  return RT_OK;
}

int rt_net_save(const rt_net* net, const char* path) {
  if (!net || !path) return fail(RT_ERR_INVALID_ARG, "net or path is NULL");
  const size_t n = rt::nn::kParams;
  std::vector<unsigned char> buf(kCkptHeader + 3 * n * 4 + 4);
  unsigned char* p = buf.data();
  std::memcpy(p, kCkptMagic, 8);
  const uint32_t head[4] = {kCkptVersion, (uint32_t)n, net->step, net->fp8 ? 1u : 0u};
  std::memcpy(p + 8, head, sizeof head);
  std::memcpy(p + 24, net->act_scale, 3 * 4);
  cudaError_t e = cudaDeviceSynchronize();
  float* const src[3] = {net->params, net->m, net->v};
  for (int k = 0; k < 3 && e == cudaSuccess; ++k)
    e = cudaMemcpy(p + kCkptHeader + (size_t)k * n * 4, src[k], n * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "rt_net_save: download");
  const uint32_t crc = crc32(p, buf.size() - 4);
  std::memcpy(p + buf.size() - 4, &crc, 4);
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(RT_ERR_INVALID_ARG, std::string("rt_net_save: cannot open ") + path);
  const bool ok = std::fwrite(p, 1, buf.size(), f) == buf.size();
  if (std::fclose(f) != 0 || !ok) return fail(RT_ERR_INVALID_ARG, std::string("rt_net_save: write failed: ") + path);
  return RT_OK;
}

int rt_net_load(const char* path, rt_net** out) {
  if (!path || !out) return fail(RT_ERR_INVALID_ARG, "path or out is NULL");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(RT_ERR_INVALID_ARG, std::string("rt_net_load: cannot open ") + path);
  const size_t n = rt::nn::kParams, want = kCkptHeader + 3 * n * 4 + 4;
  std::vector<unsigned char> buf(want + 1);
  const size_t got = std::fread(buf.data(), 1, buf.size(), f);
  std::fclose(f);
  const unsigned char* p = buf.data();
  if (got != want || std::memcmp(p, kCkptMagic, 8) != 0)
    return fail(RT_ERR_INVALID_ARG, std::string("rt_net_load: not a network checkpoint (or wrong size): ") + path);
  uint32_t head[4], crc = 0;
  std::memcpy(head, p + 8, sizeof head);
  std::memcpy(&crc, p + want - 4, 4);
  if (head[0] != kCkptVersion || head[1] != n || head[3] > 1)
    return fail(RT_ERR_INVALID_ARG, "rt_net_load: unsupported checkpoint version or parameter count");
  if (crc32(p, want - 4) != crc) return fail(RT_ERR_INVALID_ARG, "rt_net_load: CRC mismatch");
  std::vector<float> params(n), m(n), v(n);
  std::memcpy(params.data(), p + kCkptHeader, n * 4);
  std::memcpy(m.data(), p + kCkptHeader + n * 4, n * 4);
  std::memcpy(v.data(), p + kCkptHeader + 2 * n * 4, n * 4);
  float act[3];
  std::memcpy(act, p + 24, sizeof act);
  rt_net* net = nullptr;
  int rc = rt_net_create(params.data(), (uint32_t)n, &net);
  if (rc) return rc;
  cudaError_t e = cudaMemcpy(net->m, m.data(), n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(net->v, v.data(), n * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { rt_net_destroy(net); return cuda_fail(e, "rt_net_load: upload"); }
  net->step = head[2];
  if (head[3]) {
    rc = rt_net_set_fp8(net, act);
    if (rc) { rt_net_destroy(net); return rc; }
  }
  *out = net;
  return RT_OK;
}

int rt_net_forward(rt_net* net, const uint16_t* d_feat16, uint32_t W, uint32_t H, float* d_prob,
                   void* cuda_stream) {
  if (!net || !d_feat16 || !d_prob || W < 1 || H < 1) return fail(RT_ERR_INVALID_ARG, "bad argument");
  if ((uint64_t)W * H > (1ull << 30)) return fail(RT_ERR_INVALID_ARG, "image too large");
  int rc = net_buffers(net, (uint64_t)W * H);
  if (rc) return rc;
  cudaError_t e = net_forward(net, reinterpret_cast<const __nv_bfloat16*>(d_feat16), net->act, d_prob,
                              W, H, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(e, "network forward");
  return RT_OK;
}

int rt_net_forward_images(rt_net* net, const uint16_t* d_feat16, uint32_t n_img, uint32_t W, uint32_t H,
                          float* d_prob, void* cuda_stream) {
  if (!net || !d_feat16 || !d_prob || n_img < 1 || W < 1 || H < 1) return fail(RT_ERR_INVALID_ARG, "bad argument");
  if ((uint64_t)W * H * n_img > (1ull << 30)) return fail(RT_ERR_INVALID_ARG, "images too large");
  int rc = net_buffers(net, (uint64_t)W * H * n_img);
  if (rc) return rc;
  cudaError_t e = net_forward(net, reinterpret_cast<const __nv_bfloat16*>(d_feat16), net->act, d_prob,
                              W, H, static_cast<cudaStream_t>(cuda_stream), n_img);
  if (e != cudaSuccess) return cuda_fail(e, "network forward (images)");
  return RT_OK;
}

int rt_net_train_step(rt_net* net, const uint16_t* d_feat16, const float* d_label, uint32_t W,
                      uint32_t H, float lr, float* host_loss, float* d_grads, void* cuda_stream) {
  if (!net || !d_feat16 || !d_label || W < 1 || H < 1 || !(lr >= 0.f) || !std::isfinite(lr))
    return fail(RT_ERR_INVALID_ARG, "bad argument");
  if ((uint64_t)W * H > (1ull << 30)) return fail(RT_ERR_INVALID_ARG, "image too large");
  const uint64_t P = (uint64_t)W * H;
  int rc = net_buffers(net, P);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const __nv_bfloat16* f16 = reinterpret_cast<const __nv_bfloat16*>(d_feat16);
  cudaError_t e = rt::nn::forward(f16, net->params, net->wf, net->act[0], net->act[1], net->act[2],
                                  net->prob, W, H, net->err, st);
  if (e == cudaSuccess)
    e = rt::nn::backward(f16, d_label, net->wb, net->act[0], net->act[1], net->act[2], net->prob,
                         net->g16, net->g32, net->dz[0], net->dz[1], net->wpart, net->grads,
                         net->loss, W, H, net->err, st);
  if (e == cudaSuccess && d_grads)
    e = cudaMemcpyAsync(d_grads, net->grads, (size_t)rt::nn::kParams * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && lr > 0.f) {
    net->step += 1;
    e = rt::nn::adam(net->params, net->grads, net->m, net->v, rt::nn::kParams, lr, net->step, st);
    if (e == cudaSuccess) e = rt::nn::pack_weights(net->params, net->wf, net->wb, st);
  }
  if (e == cudaSuccess && host_loss) {
    float sum = 0.f;
    e = cudaMemcpyAsync(&sum, net->loss, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    *host_loss = sum / (float)P;
  }
  if (e != cudaSuccess) return cuda_fail(e, "network training step");
  return RT_OK;
}

int rt_reproj_warp(const float* d_depth_L, const float* d_normal_L, const uint32_t* d_id_L,
                   const float* d_rgb_L, const float* d_refl_L, uint32_t W, uint32_t H, float f_px, float eye_sep,
                   float convergence, uint64_t* d_zbuf, uint16_t* d_feat16, float* d_feat32,
                   uint8_t* d_hole, float* d_warped, void* cuda_stream) {
  if (!d_depth_L || !d_normal_L || !d_id_L || !d_rgb_L || !d_zbuf || W < 1 || H < 1)
    return fail(RT_ERR_INVALID_ARG, "bad argument");
  if ((uint64_t)W * H > (1ull << 31)) return fail(RT_ERR_INVALID_ARG, "image too large");
  if (!(f_px > 0.f) || !(eye_sep >= 0.f) || !(convergence > 0.f) || !std::isfinite(f_px) ||
      !std::isfinite(eye_sep) || !std::isfinite(convergence))
    return fail(RT_ERR_INVALID_ARG, "f_px, eye_sep, convergence out of range");
  cudaError_t e = rt::reproj_warp(d_depth_L, d_normal_L, d_id_L, d_rgb_L, d_refl_L, W, H, f_px, eye_sep,
                                  convergence, reinterpret_cast<unsigned long long*>(d_zbuf),
                                  reinterpret_cast<__nv_bfloat16*>(d_feat16), d_feat32, d_hole,
                                  d_warped, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(e, "warp");
  return RT_OK;
}

int rt_reproj_training_pair(const rt_scene* scene, const rt_camera* cam, float eye_sep,
                            float convergence, uint32_t W, uint32_t H, uint32_t max_depth,
                            float* d_out_L, float* d_out_R, uint16_t* d_feat16, float* d_label,
                            float label_threshold, void* cuda_stream) {
  rt::RenderArgs a;
  int rc = rt::make_render_args(scene, cam, eye_sep, convergence, W, H, max_depth, a);
  if (rc) return rc;
  if (!d_out_L || !d_out_R || !d_feat16 || !d_label || !(label_threshold >= 0.f))
    return fail(RT_ERR_INVALID_ARG, "bad argument");
  const uint64_t P = (uint64_t)W * H;
  rc = rt::ensure_workspace(scene, W, H);
  if (!rc) rc = reproj_buffers(scene, P);
  if (rc) return rc;
  rt::ReprojBuffers& rp = const_cast<rt_scene*>(scene)->ws.rp;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  a.out_L = d_out_L; a.out_R = d_out_R;   // both eyes in full: the labels compare with the right
  a.hit_L = rp.id_L; a.depth_L = rp.depth_L; a.normal_L = rp.normal_L; a.refl_L = rp.refl_L;
  rt::profile_begin(const_cast<rt_scene*>(scene)->ws, st);
  cudaError_t e = rt::render(a, const_cast<rt_scene*>(scene)->ws, st);
  if (e == cudaSuccess)
    e = rt::reproj_warp(rp.depth_L, rp.normal_L, rp.id_L, d_out_L, rp.refl_L, W, H, focal_px(cam, H), eye_sep,
                        convergence, rp.zbuf, reinterpret_cast<__nv_bfloat16*>(d_feat16), nullptr,
                        rp.hole, rp.warped, st);
  if (e == cudaSuccess) e = rt::reproj_labels(rp.hole, rp.warped, d_out_R, (uint32_t)P, label_threshold, d_label, st);
  if (e != cudaSuccess) return cuda_fail(e, "training pair");
  return RT_OK;
}

int rt_render_stereo_reproj(const rt_scene* scene, const rt_camera* cam, float eye_sep,
                            float convergence, uint32_t W, uint32_t H, uint32_t max_depth,
                            rt_net* net, float threshold, float* d_out_L, float* d_out_R,
                            uint32_t* d_n_retraced, void* cuda_stream) {
  rt::RenderArgs a;
  int rc = rt::make_render_args(scene, cam, eye_sep, convergence, W, H, max_depth, a);
  if (rc) return rc;
  if (!d_out_L || !d_out_R || !std::isfinite(threshold)) return fail(RT_ERR_INVALID_ARG, "bad argument");
  const uint64_t P = (uint64_t)W * H;
  rc = rt::ensure_workspace(scene, W, H);
  if (!rc) rc = reproj_buffers(scene, P);
  if (!rc && net) rc = net_buffers(net, P);
  if (rc) return rc;
  rt_scene* sc = const_cast<rt_scene*>(scene);
  rt::ReprojBuffers& rp = sc->ws.rp;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // 1. left eye with its G-buffer
  rt::profile_begin(sc->ws, st);
  a.eyes = 1u;
  a.out_L = d_out_L; a.out_R = nullptr;   // the left pass resolves the left eye only
  a.hit_L = rp.id_L; a.depth_L = rp.depth_L; a.normal_L = rp.normal_L; a.refl_L = rp.refl_L;
  cudaError_t e = rt::render(a, sc->ws, st);
  // 2. forward warp to the right grid, network features
  if (e == cudaSuccess)
    e = rt::reproj_warp(rp.depth_L, rp.normal_L, rp.id_L, d_out_L, rp.refl_L, W, H, focal_px(cam, H), eye_sep,
                        convergence, rp.zbuf, net ? rp.feat16 : nullptr, nullptr, rp.hole,
                        rp.warped, st);
  rt::profile_mark(sc->ws, rt::ST_WARP, st);
  // 3. retrace probability
  if (e == cudaSuccess && net) {
    e = net_forward(net, rp.feat16, rp.act, rp.prob, W, H, st);
    rt::profile_mark(sc->ws, rt::ST_NET, st);
  }
  // 4. mask = hole, reflective source, or p > threshold, compacted
  if (e == cudaSuccess)
    e = rt::reproj_mask(rp.hole, net ? rp.prob : nullptr, (uint32_t)P, threshold, rp.mask, rp.plist,
                        rp.count, st);
  rt::profile_mark(sc->ws, rt::ST_MASK, st);
  // 5. trace the masked right pixels (count read on the device)
  if (e == cudaSuccess) {
    rt::RenderArgs b = a;
    b.eyes = 2u;
    b.hit_L = nullptr; b.depth_L = nullptr; b.normal_L = nullptr; b.refl_L = nullptr;
    b.plist = rp.plist;
    b.plist_n = 0;
    b.plist_n_dev = rp.count;
    b.resolve = false;
    b.trace_stage = rt::ST_RETRACE;
    e = rt::render(b, sc->ws, st);
  }
  // 6. compose the right image
  if (e == cudaSuccess)
    e = rt::reproj_compose(rp.mask, sc->ws.accum + 3 * P, rp.warped, (uint32_t)P,
                           1.f / sc->color_scale, d_out_R, st);
  rt::profile_mark(sc->ws, rt::ST_COMPOSE, st);
  if (e == cudaSuccess && d_n_retraced)
    e = cudaMemcpyAsync(d_n_retraced, rp.count, 4, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "reprojection render");
  return RT_OK;
}

int rt_render_stereo_reproj_frames(const rt_scene* scene, const rt_camera* cams, uint32_t n_frames,
                                   float eye_sep, float convergence, uint32_t W, uint32_t H,
                                   uint32_t max_depth, rt_net* net, float threshold, float* d_out_L,
                                   float* d_out_R, uint32_t* d_n_retraced, void* cuda_stream) {
  if (!cams || n_frames < 1 || n_frames > (uint32_t)rt::kMaxFrames)
    return fail(RT_ERR_INVALID_ARG, "need 1 <= n_frames <= RT_MAX_FRAMES cameras");
  rt::RenderArgs a;
  int rc = rt::make_render_args(scene, &cams[0], eye_sep, convergence, W, H, max_depth, a);
  if (rc) return rc;
  if (!d_out_L || !d_out_R || !std::isfinite(threshold)) return fail(RT_ERR_INVALID_ARG, "bad argument");
  const uint64_t P = (uint64_t)W * H, FP = P * n_frames;
  if (2 * FP > (1ull << 31)) return fail(RT_ERR_INVALID_ARG, "2 * n_frames * W * H exceeds 2^31");
  // every frame's camera, validated like a single render's; the warp's
  // disparity needs one focal length, so the vertical fields of view agree
  rt::CameraParams frames[rt::kMaxFrames];
  frames[0] = a.cam;
  for (uint32_t f = 1; f < n_frames; ++f) {
    if (cams[f].vfov_deg != cams[0].vfov_deg)
      return fail(RT_ERR_INVALID_ARG, "all frames need the same vfov_deg");
    rt::RenderArgs b;
    rc = rt::make_render_args(scene, &cams[f], eye_sep, convergence, W, H, max_depth, b);
    if (rc) return rc;
    frames[f] = b.cam;
  }
  rc = rt::ensure_workspace(scene, W, H * n_frames);
  if (!rc) rc = reproj_buffers(scene, FP);
  if (!rc && net) rc = net_buffers(net, FP);
  if (rc) return rc;
  rt_scene* sc = const_cast<rt_scene*>(scene);
  rt::ReprojBuffers& rp = sc->ws.rp;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  a.n_frames = n_frames;
  a.frames = frames;
  // 1. left eyes of all frames, one launch, with their G-buffers
  rt::profile_begin(sc->ws, st);
  a.eyes = 1u;
  a.out_L = d_out_L; a.out_R = nullptr;   // the left pass resolves the left eye only
  a.hit_L = rp.id_L; a.depth_L = rp.depth_L; a.normal_L = rp.normal_L; a.refl_L = rp.refl_L;
  cudaError_t e = rt::render(a, sc->ws, st);
  // 2. forward warp: it moves pixels along their row only, so the frames,
  //    stacked as one image of n_frames * H rows, warp in one pass
  if (e == cudaSuccess)
    e = rt::reproj_warp(rp.depth_L, rp.normal_L, rp.id_L, d_out_L, rp.refl_L, W, H * n_frames, focal_px(&cams[0], H),
                        eye_sep, convergence, rp.zbuf, net ? rp.feat16 : nullptr, nullptr, rp.hole,
                        rp.warped, st);
  rt::profile_mark(sc->ws, rt::ST_WARP, st);
  // 3. the network over all frames, one launch per layer (a 3x3 window never
  //    crosses from one frame into the next)
  if (e == cudaSuccess && net) {
    e = net_forward(net, rp.feat16, rp.act, rp.prob, W, H, st, n_frames);
    rt::profile_mark(sc->ws, rt::ST_NET, st);
  }
  // 4. mask over every right pixel of every frame, compacted into one list
  if (e == cudaSuccess)
    e = rt::reproj_mask(rp.hole, net ? rp.prob : nullptr, (uint32_t)FP, threshold, rp.mask, rp.plist,
                        rp.count, st);
  rt::profile_mark(sc->ws, rt::ST_MASK, st);
  // 5. the masked right pixels of all frames, one launch
  if (e == cudaSuccess) {
    rt::RenderArgs b = a;
    b.eyes = 2u;
    b.hit_L = nullptr; b.depth_L = nullptr; b.normal_L = nullptr; b.refl_L = nullptr;
    b.plist = rp.plist;
    b.plist_n = 0;
    b.plist_n_dev = rp.count;
    b.resolve = false;
    b.trace_stage = rt::ST_RETRACE;
    e = rt::render(b, sc->ws, st);
  }
  // 6. right images of all frames
  if (e == cudaSuccess)
    e = rt::reproj_compose(rp.mask, sc->ws.accum + 3 * FP, rp.warped, (uint32_t)FP,
                           1.f / sc->color_scale, d_out_R, st);
  rt::profile_mark(sc->ws, rt::ST_COMPOSE, st);
  if (e == cudaSuccess && d_n_retraced)
    e = cudaMemcpyAsync(d_n_retraced, rp.count, 4, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "multi-frame reprojection render");
  return RT_OK;
}

}  // extern "C"
