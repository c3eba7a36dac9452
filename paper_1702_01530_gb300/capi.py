"""Python binding of the C-ABI in ``include/rt_stereo.h`` and
``include/rt_probes.h`` (ctypes).

Argument marshalling only: every step of BVH construction and rendering
runs in the CUDA library ``_build/librtstereo.so``. Functions keep the C
names. Device buffers are passed as CUDA torch tensors (or raw integer
device addresses); streams as ``torch.cuda.Stream``, raw handles, or None
(= torch's current stream). There is no CPU fallback: if the library is
missing, loading it raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import scenegen
from .build import INCLUDE, LIB

RT_OK = 0
RT_ERR_INVALID_ARG = -1
RT_ERR_CUDA = -2
RT_ERR_OOM = -3
RT_ERR_TIMEOUT = -4
RT_ERR_DEVICE_CHECK = -5
RT_MISS_ID = 0xFFFFFFFF
HEADER = os.path.join(INCLUDE, "rt_stereo.h")

_lib = None
_vp = ctypes.c_void_p
_u32 = ctypes.c_uint32
_f32 = ctypes.c_float


class RtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rt error {code}: {msg}")
        self.code = code


_SIGS = {
    "rt_scene_create": (ctypes.c_int, [_vp, _u32, _vp, _u32, _vp, _u32, _vp, _u32, _vp,
                                       ctypes.POINTER(_vp)]),
    "rt_scene_destroy": (None, [_vp]),
    "rt_render_stereo": (ctypes.c_int, [_vp, _vp, _f32, _f32, _u32, _u32, _u32, _vp, _vp, _vp]),
    "rt_render_stereo_aux": (ctypes.c_int, [_vp, _vp, _f32, _f32, _u32, _u32, _u32, _vp, _vp,
                                            _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "rt_render_stereo_sequence": (ctypes.c_int, [_vp, _vp, _u32, _f32, _f32, _u32, _u32, _u32,
                                                 _vp, _vp, _vp]),
    "rt_render_stereo_host": (ctypes.c_int, [_vp, _vp, _f32, _f32, _u32, _u32, _u32, _vp, _vp,
                                             _vp]),
    "rt_render_stereo_rows": (ctypes.c_int, [_vp, _vp, _f32, _f32, _u32, _u32, _u32, _u32, _u32,
                                             _vp, _vp, _vp, _vp]),
    "rt_sync_status": (ctypes.c_int, [_vp, _vp]),
    "rt_scene_get_bvh": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "rt_scene_num_prims": (_u32, [_vp]),
    "rt_debug_set_pool_capacity": (ctypes.c_int, [_vp, _u32]),
    "rt_debug_get_sah_tree": (ctypes.c_int, [_vp, _vp]),
    "rt_debug_set_sah_slicing": (ctypes.c_int, [ctypes.c_int]),
    "rt_debug_set_node": (ctypes.c_int, [_vp, _u32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int]),
    "rt_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
    "rt_scene_set_traversal": (ctypes.c_int, [_vp, ctypes.c_int]),
    "rt_profile_read": (ctypes.c_int, [_vp, _vp]),
    "rt_build_lbvh_noalloc": (ctypes.c_int, [_vp, _u32, _vp, _u32, _vp, _vp, _vp, _vp, _vp]),
    "rt_net_create": (ctypes.c_int, [_vp, _u32, ctypes.POINTER(_vp)]),
    "rt_net_destroy": (None, [_vp]),
    "rt_net_get_params": (ctypes.c_int, [_vp, _vp]),
    "rt_net_status": (ctypes.c_int, [_vp, _vp]),
    "rt_net_forward": (ctypes.c_int, [_vp, _vp, _u32, _u32, _vp, _vp]),
    "rt_net_set_fp8": (ctypes.c_int, [_vp, _vp]),
    "rt_net_forward_images": (ctypes.c_int, [_vp, _vp, _u32, _u32, _u32, _vp, _vp]),
    "rt_net_activation_amax": (ctypes.c_int, [_vp, _vp, _u32, _u32, _vp, _vp]),
    "rt_net_calibrate_fp8": (ctypes.c_int, [_vp, _vp, _u32, _u32, _u32, _vp, _vp, _vp]),
    "rt_net_save": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "rt_net_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_vp)]),
    "rt_net_train_step": (ctypes.c_int, [_vp, _vp, _vp, _u32, _u32, _f32, _vp, _vp, _vp]),
    "rt_reproj_warp": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _u32, _u32, _f32, _f32, _f32, _vp,
                                      _vp, _vp, _vp, _vp, _vp]),
    "rt_reproj_training_pair": (ctypes.c_int, [_vp, _vp, _f32, _f32, _u32, _u32, _u32, _vp, _vp,
                                               _vp, _vp, _f32, _vp]),
    "rt_render_stereo_reproj": (ctypes.c_int, [_vp, _vp, _f32, _f32, _u32, _u32, _u32, _vp, _f32,
                                               _vp, _vp, _vp, _vp]),
    "rt_render_stereo_reproj_frames": (ctypes.c_int, [_vp, _vp, _u32, _f32, _f32, _u32, _u32, _u32,
                                                      _vp, _f32, _vp, _vp, _vp, _vp]),
    "rt_stereo_composite": (ctypes.c_int, [_vp, _vp, _u32, _u32, ctypes.c_int, _vp, _vp]),
    "rt_batch_create": (ctypes.c_int, [_vp, _u32, _vp, ctypes.POINTER(_vp)]),
    "rt_batch_destroy": (None, [_vp]),
    "rt_batch_launch": (ctypes.c_int, [_vp, _vp]),
    "rt_batch_set_camera": (ctypes.c_int, [_vp, _u32, _vp, _f32, _f32]),
    "rt_batch_autotune": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp]),
    "rt_batch_stats": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "rt_probe_l2_read": (ctypes.c_int, [_vp, ctypes.c_uint64, _u32, _vp, ctypes.c_uint64, _vp]),
    "rt_probe_l2_threads": (ctypes.c_uint64, []),
    "rt_probe_mufu": (ctypes.c_int, [_u32, _vp, ctypes.c_uint64, _vp]),
    "rt_probe_mufu_threads": (ctypes.c_uint64, []),
    "rt_last_error": (ctypes.c_char_p, []),
    "rt_version": (ctypes.c_char_p, []),
}


def library_path() -> str:
    return LIB


def lib():
    """Load librtstereo.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"{LIB} is missing: build it with "
                              "`python -m paper_1702_01530_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the functions declared in include/*.h."""
    import glob
    src = "".join(open(h).read() for h in sorted(glob.glob(os.path.join(INCLUDE, "*.h"))))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z0-9_]+)\s*\(", src)))


def rt_last_error() -> str:
    return lib().rt_last_error().decode()


def rt_version() -> str:
    return lib().rt_version().decode()


def _check(rc: int):
    if rc != RT_OK:
        raise RtError(rc, rt_last_error())


def _dptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("device buffers must be contiguous CUDA tensors")
    return x.data_ptr()


def _stream(s):
    if s is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
        except ImportError:
            return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _np(a, dt):
    a = np.ascontiguousarray(a, dtype=dt)
    return a, (a.ctypes.data if a.size else None)


def rt_scene_create(spheres, triangles, materials, lights, stream=None) -> int:
    sp, psp = _np(spheres, scenegen.SPHERE_DT)
    tr, ptr = _np(triangles, scenegen.TRIANGLE_DT)
    mt, pmt = _np(materials, scenegen.MATERIAL_DT)
    li, pli = _np(lights, scenegen.LIGHT_DT)
    h = _vp()
    _check(lib().rt_scene_create(psp, len(sp), ptr, len(tr), pmt, len(mt), pli, len(li),
                                 _stream(stream), ctypes.byref(h)))
    return h.value


def rt_scene_destroy(scene: int):
    lib().rt_scene_destroy(scene)


def _cam(camera):
    c = np.ascontiguousarray(np.asarray(camera, dtype=scenegen.CAMERA_DT).reshape(()))
    return c, c.ctypes.data


def rt_render_stereo(scene, camera, eye_sep, convergence, W, H, max_depth, out_L, out_R,
                     stream=None):
    c, pc = _cam(camera)
    _check(lib().rt_render_stereo(scene, pc, eye_sep, convergence, W, H, max_depth, _dptr(out_L),
                                  _dptr(out_R), _stream(stream)))


def rt_render_stereo_aux(scene, camera, eye_sep, convergence, W, H, max_depth, out_L, out_R,
                         hit_id_L=None, hit_id_R=None, depth_L=None, depth_R=None,
                         ray_counts=None, work=None, stream=None):
    c, pc = _cam(camera)
    _check(lib().rt_render_stereo_aux(scene, pc, eye_sep, convergence, W, H, max_depth,
                                      _dptr(out_L), _dptr(out_R), _dptr(hit_id_L),
                                      _dptr(hit_id_R), _dptr(depth_L), _dptr(depth_R),
                                      _dptr(ray_counts), _dptr(work), _stream(stream)))


def rt_render_stereo_rows(scene, camera, eye_sep, convergence, W, H, max_depth, row0, n_rows,
                          out_L, out_R, ray_counts=None, stream=None):
    """Rows row0 .. row0 + n_rows - 1 of both eyes of the W x H pair into
    band buffers of n_rows x W x 3 float32 each."""
    c, pc = _cam(camera)
    _check(lib().rt_render_stereo_rows(scene, pc, eye_sep, convergence, W, H, max_depth, row0,
                                       n_rows, _dptr(out_L), _dptr(out_R), _dptr(ray_counts),
                                       _stream(stream)))


def _hptr(x):
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous or x.dtype != np.float32:
            raise ValueError("host buffers must be contiguous float32")
        return x.ctypes.data
    if x.is_cuda or not x.is_contiguous():
        raise ValueError("host buffers must be contiguous CPU tensors")
    return x.data_ptr()


def rt_render_stereo_host(scene, camera, eye_sep, convergence, W, H, max_depth, host_L, host_R,
                          stream=None):
    c, pc = _cam(camera)
    _check(lib().rt_render_stereo_host(scene, pc, eye_sep, convergence, W, H, max_depth,
                                       _hptr(host_L), _hptr(host_R), _stream(stream)))


def rt_render_stereo_sequence(scene, cameras, eye_sep, convergence, W, H, max_depth, hosts_L,
                              hosts_R, stream=None):
    """One stereo pair per camera into host buffers hosts_L[f], hosts_R[f]
    (H*W*3 float32 each; a buffer may repeat), copies overlapped with the
    next frame's render."""
    cams = np.ascontiguousarray(np.asarray(cameras, dtype=scenegen.CAMERA_DT).reshape(-1))
    n = cams.shape[0]
    if len(hosts_L) != n or len(hosts_R) != n:
        raise ValueError("one left and one right host buffer per camera")
    pl = (ctypes.c_void_p * max(1, n))(*[_hptr(x) for x in hosts_L])
    pr = (ctypes.c_void_p * max(1, n))(*[_hptr(x) for x in hosts_R])
    _check(lib().rt_render_stereo_sequence(scene, cams.ctypes.data, n, eye_sep, convergence, W, H,
                                           max_depth, ctypes.cast(pl, ctypes.c_void_p),
                                           ctypes.cast(pr, ctypes.c_void_p), _stream(stream)))


def rt_sync_status(scene, stream=None):
    _check(lib().rt_sync_status(scene, _stream(stream)))


def rt_debug_set_node(scene, node, left, right, empty_right=False):
    _check(lib().rt_debug_set_node(scene, node, left, right, int(bool(empty_right))))


def rt_debug_set_pool_capacity(scene, entries):
    _check(lib().rt_debug_set_pool_capacity(scene, entries))


def rt_debug_get_sah_tree(scene) -> np.ndarray:
    """The SAH render tree as (n-1, 16) uint32 words (boxes as FP32 bits)."""
    n = rt_scene_num_prims(scene)
    out = np.zeros((max(n - 1, 1), 16), np.uint32)
    _check(lib().rt_debug_get_sah_tree(scene, out.ctypes.data))
    return out[:max(n - 1, 0)]


def rt_debug_set_sah_slicing(enable):
    _check(lib().rt_debug_set_sah_slicing(int(bool(enable))))


STAGES = ("clear", "trace", "resolve", "warp", "net", "mask", "retrace", "compose")


RT_TREE_SAH, RT_TREE_WIDE, RT_TREE_LBVH = 0, 1, 2


def rt_scene_set_traversal(scene, tree=RT_TREE_WIDE):
    """Tree the scene's renders walk: RT_TREE_SAH (default), RT_TREE_WIDE
    or RT_TREE_LBVH (booleans map True -> RT_TREE_WIDE, False -> RT_TREE_SAH)."""
    if isinstance(tree, bool):
        tree = RT_TREE_WIDE if tree else RT_TREE_SAH
    _check(lib().rt_scene_set_traversal(scene, int(tree)))


def rt_profile_enable(scene, on=True):
    _check(lib().rt_profile_enable(scene, int(bool(on))))


def rt_profile_read(scene) -> dict:
    ms = np.zeros(len(STAGES), np.float32)
    _check(lib().rt_profile_read(scene, ms.ctypes.data))
    return dict(zip(STAGES, ms.astype(float).tolist()))


def rt_scene_num_prims(scene) -> int:
    return lib().rt_scene_num_prims(scene)


def rt_scene_get_bvh(scene) -> dict:
    n = rt_scene_num_prims(scene)
    keys = np.zeros(n, np.uint64)
    left = np.zeros(max(n - 1, 0), np.int32)
    right = np.zeros(max(n - 1, 0), np.int32)
    parent = np.zeros(2 * n - 1, np.int32)
    ibox = np.zeros((max(n - 1, 0), 6), np.float32)
    lbox = np.zeros((n, 6), np.float32)
    p = lambda a: a.ctypes.data if a.size else None  # noqa: E731
    _check(lib().rt_scene_get_bvh(scene, p(keys), p(left), p(right), p(parent), p(ibox),
                                  p(lbox)))
    return dict(keys=keys, left=left, right=right, parent=parent, inner_box=ibox, leaf_box=lbox)


def rt_build_lbvh_noalloc(d_spheres, n_spheres, d_tris, n_tris, d_nodes, d_prims, d_keys,
                          d_parent, stream=None):
    """LBVH build into caller-owned device buffers with no device allocation
    (for callers that may not call cudaMalloc); see include/rt_stereo.h."""
    _check(lib().rt_build_lbvh_noalloc(_dptr(d_spheres), n_spheres, _dptr(d_tris), n_tris,
                                       _dptr(d_nodes), _dptr(d_prims), _dptr(d_keys),
                                       _dptr(d_parent), _stream(stream)))


COMPOSITE_ANAGLYPH_COLOR, COMPOSITE_ANAGLYPH_GRAY, COMPOSITE_SIDE_BY_SIDE = 0, 1, 2


# ------------------------------------------------------------- batching
RT_BATCH_MAX_REQUESTS = 4096
RT_BATCH_ORDER_GIVEN, RT_BATCH_ORDER_LARGEST_FIRST, RT_BATCH_ORDER_SMALLEST_FIRST = 0, 1, 2
REQUEST_DT = np.dtype({"names": ["scene", "camera", "eye_sep", "convergence", "W", "H",
                                 "max_depth", "reserved", "d_out_L", "d_out_R"],
                       "formats": ["<u8", scenegen.CAMERA_DT, "<f4", "<f4", "<u4", "<u4", "<u4",
                                   "<u4", "<u8", "<u8"],
                       "offsets": [0, 8, 48, 52, 56, 60, 64, 68, 72, 80], "itemsize": 88})
BATCH_CONFIG_DT = np.dtype([(k, "<u4") for k in ("tile_w", "tile_h", "blocks_per_sm", "cap_r",
                                                  "order", "track_latency")])


def batch_config(tile_w=4, tile_h=4, blocks_per_sm=0, cap_r=64, order=RT_BATCH_ORDER_LARGEST_FIRST,
                 track_latency=1) -> np.ndarray:
    c = np.zeros(1, BATCH_CONFIG_DT)
    for k, v in dict(tile_w=tile_w, tile_h=tile_h, blocks_per_sm=blocks_per_sm, cap_r=cap_r,
                     order=order, track_latency=track_latency).items():
        c[k] = v
    return c


def make_requests(items) -> np.ndarray:
    """items: (scene handle, camera record, eye_sep, convergence, W, H,
    max_depth, out_L, out_R) per request; outputs are CUDA tensors or device
    addresses."""
    r = np.zeros(len(items), REQUEST_DT)
    for i, (h, cam, es, cv, W, H, D, oL, oR) in enumerate(items):
        r["scene"][i] = h or 0
        r["camera"][i] = np.asarray(cam, scenegen.CAMERA_DT).reshape(())
        r["eye_sep"][i], r["convergence"][i] = es, cv
        r["W"][i], r["H"][i], r["max_depth"][i] = W, H, D
        r["d_out_L"][i] = _dptr(oL) or 0
        r["d_out_R"][i] = _dptr(oR) or 0
    return r


def rt_batch_create(reqs: np.ndarray, cfg: np.ndarray | None = None):
    reqs = np.ascontiguousarray(reqs, REQUEST_DT)
    out = _vp()
    c = None if cfg is None else np.ascontiguousarray(cfg, BATCH_CONFIG_DT)
    _check(lib().rt_batch_create(reqs.ctypes.data if len(reqs) else None, len(reqs),
                                 None if c is None else c.ctypes.data, ctypes.byref(out)))
    return out.value


def rt_batch_destroy(b):
    lib().rt_batch_destroy(b)


def rt_batch_launch(b, stream=None):
    _check(lib().rt_batch_launch(b, _stream(stream)))


def rt_batch_set_camera(b, i, cam, eye_sep, convergence):
    c = np.ascontiguousarray(np.asarray(cam, scenegen.CAMERA_DT).reshape(1))
    _check(lib().rt_batch_set_camera(b, i, c.ctypes.data, eye_sep, convergence))


def rt_batch_autotune(b, reps=3, stream=None):
    c = np.zeros(1, BATCH_CONFIG_DT)
    ms = ctypes.c_float()
    _check(lib().rt_batch_autotune(b, reps, _stream(stream), c.ctypes.data, ctypes.byref(ms)))
    return c, ms.value


def rt_batch_stats(b, n_requests):
    rays = np.zeros(3, np.uint64)
    lat = np.zeros(n_requests, np.float32)
    c = np.zeros(1, BATCH_CONFIG_DT)
    _check(lib().rt_batch_stats(b, rays.ctypes.data, lat.ctypes.data, c.ctypes.data))
    return rays, lat, c


def rt_probe_l2_read(buf, n_vec, reps, sink, stream=None):
    n_sink = sink.numel() * sink.element_size() // 16
    _check(lib().rt_probe_l2_read(_dptr(buf), n_vec, reps, _dptr(sink), n_sink, _stream(stream)))


def rt_probe_l2_threads() -> int:
    return int(lib().rt_probe_l2_threads())


def rt_probe_mufu(iters, sink, stream=None):
    _check(lib().rt_probe_mufu(iters, _dptr(sink), sink.numel(), _stream(stream)))


def rt_probe_mufu_threads() -> int:
    return int(lib().rt_probe_mufu_threads())


def rt_stereo_composite(L, R, W, H, mode, out, stream=None):
    _check(lib().rt_stereo_composite(_dptr(L), _dptr(R), W, H, mode, _dptr(out), _stream(stream)))


RT_NET_PARAMS = 21697


def rt_net_create(params) -> int:
    p = np.ascontiguousarray(params, np.float32).reshape(-1)
    h = _vp()
    _check(lib().rt_net_create(p.ctypes.data, len(p), ctypes.byref(h)))
    return h.value


def rt_net_destroy(net):
    lib().rt_net_destroy(net)


def rt_net_get_params(net) -> np.ndarray:
    out = np.zeros(RT_NET_PARAMS, np.float32)
    _check(lib().rt_net_get_params(net, out.ctypes.data))
    return out


def rt_net_status(net, stream=None):
    _check(lib().rt_net_status(net, _stream(stream)))


def rt_net_forward(net, feat16, W, H, prob, stream=None):
    _check(lib().rt_net_forward(net, _dptr(feat16), W, H, _dptr(prob), _stream(stream)))


def rt_net_forward_images(net, feat16, n_img, W, H, prob, stream=None):
    _check(lib().rt_net_forward_images(net, _dptr(feat16), n_img, W, H, _dptr(prob), _stream(stream)))


def rt_net_set_fp8(net, act_scales):
    """act_scales: three powers of two, or None to return to BF16 inference."""
    if act_scales is None:
        _check(lib().rt_net_set_fp8(net, None))
        return
    a = np.ascontiguousarray(act_scales, np.float32)
    _check(lib().rt_net_set_fp8(net, a.ctypes.data))


def rt_net_activation_amax(net, feat16, W, H, stream=None) -> np.ndarray:
    out = np.zeros(3, np.float32)
    _check(lib().rt_net_activation_amax(net, _dptr(feat16), W, H, out.ctypes.data, _stream(stream)))
    return out


def rt_net_calibrate_fp8(net, feats, W, H, stream=None):
    """Run the BF16 network on every feature map in ``feats``, choose the FP8
    activation scales in the library and switch the network to FP8.
    Returns (amax, scales), three floats each."""
    ptrs = (ctypes.c_void_p * max(1, len(feats)))(*[_dptr(f) for f in feats])
    amax = np.zeros(3, np.float32)
    scales = np.zeros(3, np.float32)
    _check(lib().rt_net_calibrate_fp8(net, ctypes.cast(ptrs, ctypes.c_void_p), len(feats), W, H,
                                      amax.ctypes.data, scales.ctypes.data, _stream(stream)))
    return amax, scales


def rt_net_save(net, path):
    _check(lib().rt_net_save(net, os.fsencode(path)))


def rt_net_load(path) -> int:
    h = _vp()
    _check(lib().rt_net_load(os.fsencode(path), ctypes.byref(h)))
    return h.value


def rt_net_train_step(net, feat16, label, W, H, lr, want_loss=True, grads=None, stream=None):
    loss = ctypes.c_float()
    _check(lib().rt_net_train_step(net, _dptr(feat16), _dptr(label), W, H, lr,
                                   ctypes.byref(loss) if want_loss else None, _dptr(grads),
                                   _stream(stream)))
    return loss.value if want_loss else None


def rt_reproj_warp(depth_L, normal_L, id_L, rgb_L, W, H, f_px, eye_sep, convergence, zbuf,
                   feat16=None, feat32=None, hole=None, warped=None, stream=None, refl_L=None):
    _check(lib().rt_reproj_warp(_dptr(depth_L), _dptr(normal_L), _dptr(id_L), _dptr(rgb_L),
                                _dptr(refl_L), W, H,
                                f_px, eye_sep, convergence, _dptr(zbuf), _dptr(feat16),
                                _dptr(feat32), _dptr(hole), _dptr(warped), _stream(stream)))


def rt_reproj_training_pair(scene, camera, eye_sep, convergence, W, H, max_depth, out_L, out_R,
                            feat16, label, label_threshold=1e-2, stream=None):
    c, pc = _cam(camera)
    _check(lib().rt_reproj_training_pair(scene, pc, eye_sep, convergence, W, H, max_depth,
                                         _dptr(out_L), _dptr(out_R), _dptr(feat16), _dptr(label),
                                         label_threshold, _stream(stream)))


def rt_render_stereo_reproj(scene, camera, eye_sep, convergence, W, H, max_depth, net, threshold,
                            out_L, out_R, n_retraced=None, stream=None):
    c, pc = _cam(camera)
    _check(lib().rt_render_stereo_reproj(scene, pc, eye_sep, convergence, W, H, max_depth, net,
                                         threshold, _dptr(out_L), _dptr(out_R), _dptr(n_retraced),
                                         _stream(stream)))


RT_MAX_FRAMES = 8


def rt_render_stereo_reproj_frames(scene, cameras, eye_sep, convergence, W, H, max_depth, net,
                                   threshold, out_L, out_R, n_retraced=None, stream=None):
    """Learned reprojection of len(cameras) <= RT_MAX_FRAMES frames in one
    pass; out_L / out_R hold (frames, H, W, 3) float32 each."""
    cams = np.ascontiguousarray(np.asarray(cameras, dtype=scenegen.CAMERA_DT).reshape(-1))
    _check(lib().rt_render_stereo_reproj_frames(scene, cams.ctypes.data, len(cams), eye_sep,
                                                convergence, W, H, max_depth, net, threshold,
                                                _dptr(out_L), _dptr(out_R), _dptr(n_retraced),
                                                _stream(stream)))


def focal_px(camera, H) -> float:
    """f_px = (H/2)/tan(vfov/2), rounded to float32 as the library does."""
    import math
    v = float(np.asarray(camera, dtype=scenegen.CAMERA_DT)["vfov_deg"])
    return float(np.float32(0.5 * H / math.tan(0.5 * v * math.pi / 180.0)))


class Net:
    """Owns one rt_net."""

    def __init__(self, params):
        self.handle = rt_net_create(params)

    def close(self):
        if getattr(self, "handle", None):
            rt_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        return rt_net_get_params(self.handle)


class GpuScene:
    """Owns one rt_scene built from a ``scenegen.Scene``."""

    def __init__(self, scene: scenegen.Scene, stream=None):
        self.scene = scene
        self.handle = rt_scene_create(scene.spheres, scene.triangles, scene.materials,
                                      scene.lights, stream)

    def close(self):
        if getattr(self, "handle", None):
            rt_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def render(self, W=None, H=None, max_depth=None, eye_sep=None, convergence=None, aux=False,
               count_work=False, stream=None, out=None):
        """Render both eyes into (2, H, W, 3) float32 CUDA tensors (left, right)."""
        import torch
        s = self.scene
        W = s.W if W is None else W
        H = s.H if H is None else H
        D = s.max_depth if max_depth is None else max_depth
        es = s.eye_sep if eye_sep is None else eye_sep
        cv = s.convergence if convergence is None else convergence
        dev = torch.device("cuda")
        img = out if out is not None else torch.empty((2, H, W, 3), dtype=torch.float32, device=dev)
        res = {"rgb": img}
        if aux or count_work:
            hit = torch.empty((2, H, W), dtype=torch.int32, device=dev)
            dep = torch.empty((2, H, W), dtype=torch.float32, device=dev)
            rays = torch.zeros(3, dtype=torch.int64, device=dev)
            work = torch.zeros(9, dtype=torch.int64, device=dev) if count_work else None
            rt_render_stereo_aux(self.handle, s.camera, es, cv, W, H, D, img[0], img[1],
                                 hit[0], hit[1], dep[0], dep[1], rays, work, stream)
            res.update(hit_id=hit, depth=dep, rays=rays, work=work)
        else:
            rt_render_stereo(self.handle, s.camera, es, cv, W, H, D, img[0], img[1], stream)
        return res
