"""FP64 CPU oracle for the stereo ray tracer -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package. It shares no code with the CUDA path: it is a
plain FP64 C tracer (``oracle.c``) plus this ctypes wrapper. Both sides only
consume the same seeded scene arrays from ``paper_1702_01530_gb300.scenegen``.

What each function follows is stated in ``oracle.c``; in short:
``render`` is reverse ray tracing of both eyes of an off-axis stereo pair
(Sec. 2-3 of the paper: two projections from two cameras, left and right
channel independent; Table 1 "classical" ray tracing with shadow and
reflection rays), ``lbvh`` is the linear-BVH definition (Morton keys and
the binary radix tree over them), ``closest`` is a single closest-hit query.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
# ORACLE_LIB points the wrapper at another build of oracle.c (the mutation
# test loads deliberately broken copies this way)
_LIB_PATH = os.environ.get("ORACLE_LIB") or os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

MISS_ID = 0xFFFFFFFF


def build(force: bool = False, src: str = _SRC, out: str | None = None) -> str:
    """Compile oracle.c (or ``src``) with gcc: FP64, no FMA contraction."""
    if out is not None:
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                        "-pthread", src, "-o", out, "-lm"], check=True)
        return out
    if os.environ.get("ORACLE_LIB"):
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-Wall", "-shared",
                        "-fPIC", "-pthread", _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int), ("max_depth", ctypes.c_int),
                ("mode", ctypes.c_int), ("n_threads", ctypes.c_int),
                ("eye_sep", ctypes.c_double), ("convergence", ctypes.c_double),
                ("pixels", ctypes.c_void_p), ("n_pixels", ctypes.c_int64)]


class _Out(ctypes.Structure):
    _fields_ = [("rgb", ctypes.c_void_p), ("hit_id", ctypes.c_void_p), ("depth", ctypes.c_void_p),
                ("flags", ctypes.c_void_p), ("rays", ctypes.c_void_p), ("work", ctypes.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.oracle_scene_new.restype = ctypes.c_void_p
        _lib.oracle_scene_new.argtypes = [ctypes.c_void_p, ctypes.c_uint32] * 4
        _lib.oracle_scene_free.argtypes = [ctypes.c_void_p]
        _lib.oracle_lbvh.argtypes = [ctypes.c_void_p] * 7
        _lib.oracle_closest.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]
        _lib.oracle_render.argtypes = [ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(_Params), ctypes.POINTER(_Out)]
        _lib.oracle_primary_ray.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        _lib.oracle_morton30.restype = ctypes.c_uint32
        _lib.oracle_morton30.argtypes = [ctypes.c_uint32] * 3
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data if a is not None and a.size else None


def default_threads() -> int:
    return os.cpu_count() or 1


class OracleScene:
    """The oracle's view of one scene (arrays are kept alive here)."""

    MODE_AUTO, MODE_BRUTE, MODE_BVH = 0, 1, 2

    def __init__(self, scene):
        self.scene = scene
        self._arrs = [np.ascontiguousarray(a) for a in
                      (scene.spheres, scene.triangles, scene.materials, scene.lights)]
        sp, tr, mt, li = self._arrs
        self.n = len(sp) + len(tr)
        self._h = lib().oracle_scene_new(_ptr(sp), len(sp), _ptr(tr), len(tr), _ptr(mt), len(mt),
                                         _ptr(li), len(li))
        if not self._h:
            raise MemoryError("oracle_scene_new failed")
        self._cam = np.ascontiguousarray(scene.camera)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_scene_free(h)
            self._h = None

    def lbvh(self) -> dict:
        n = self.n
        keys = np.zeros(n, np.uint64)
        left = np.zeros(max(n - 1, 0), np.int32)
        right = np.zeros(max(n - 1, 0), np.int32)
        parent = np.zeros(2 * n - 1, np.int32)
        ibox = np.zeros((max(n - 1, 0), 6), np.float32)
        lbox = np.zeros((n, 6), np.float32)
        rc = lib().oracle_lbvh(self._h, _ptr(keys), _ptr(left), _ptr(right), _ptr(parent),
                               _ptr(ibox), _ptr(lbox))
        if rc:
            raise RuntimeError(f"oracle_lbvh failed ({rc})")
        return dict(keys=keys, left=left, right=right, parent=parent, inner_box=ibox, leaf_box=lbox)

    def closest(self, o, d, mode: int = 0):
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        t = ctypes.c_double()
        pid = ctypes.c_uint32()
        nt = ctypes.c_int()
        rc = lib().oracle_closest(self._h, _ptr(o), _ptr(d), mode, ctypes.byref(t),
                                  ctypes.byref(pid), ctypes.byref(nt))
        if rc:
            raise RuntimeError("oracle_closest failed")
        return t.value, pid.value, bool(nt.value)

    def render(self, W=None, H=None, max_depth=None, eye_sep=None, convergence=None,
               pixels=None, mode: int = 0, n_threads: int | None = None) -> dict:
        """Trace both eyes (or the listed pixels: index = eye*W*H + j*W + i).

        Returns rgb (n,3) float64 clamped to [0,1], hit_id (n,) uint32, depth
        (n,) float64 (view depth, inf on miss), flags (n,) uint8 (bit0: the
        primary ray is near a tie, bit1: some ray of the pixel is), rays (3,)
        primary/shadow/reflection counts, work (3,3) per ray kind: internal
        node visits, sphere tests, triangle tests (BVH mode only). Without a
        pixel list the arrays are shaped (2, H, W[, 3]) with eye 0 = left.
        """
        s = self.scene
        W = s.W if W is None else W
        H = s.H if H is None else H
        p = _Params(W, H, s.max_depth if max_depth is None else max_depth, mode,
                    n_threads or default_threads(),
                    s.eye_sep if eye_sep is None else eye_sep,
                    s.convergence if convergence is None else convergence, None, 0)
        if pixels is not None:
            pixels = np.ascontiguousarray(pixels, np.int64)
            p.pixels, p.n_pixels = _ptr(pixels), len(pixels)
            n = len(pixels)
        else:
            n = 2 * W * H
        rgb = np.zeros((n, 3), np.float64)
        hit = np.zeros(n, np.uint32)
        depth = np.zeros(n, np.float64)
        flags = np.zeros(n, np.uint8)
        rays = np.zeros(3, np.uint64)
        work = np.zeros(9, np.uint64)
        out = _Out(_ptr(rgb), _ptr(hit), _ptr(depth), _ptr(flags), _ptr(rays), _ptr(work))
        if n:
            rc = lib().oracle_render(self._h, _ptr(self._cam), ctypes.byref(p), ctypes.byref(out))
            if rc:
                raise RuntimeError(f"oracle_render failed ({rc})")
        res = dict(rgb=rgb, hit_id=hit, depth=depth, flags=flags, rays=rays, work=work.reshape(3, 3))
        if pixels is None:
            res["rgb"] = rgb.reshape(2, H, W, 3)
            for k in ("hit_id", "depth", "flags"):
                res[k] = res[k].reshape(2, H, W)
        return res


def render(scene, **kw) -> dict:
    return OracleScene(scene).render(**kw)


def morton30(qx: int, qy: int, qz: int) -> int:
    return lib().oracle_morton30(qx, qy, qz)


def primary_ray(scene, eye: int, i: int, j: int, eye_sep=None, convergence=None, W=None, H=None):
    """Origin and unit direction of pixel (i, j) of eye -1 (left) or +1 (right)."""
    cam = np.ascontiguousarray(scene.camera)
    o = np.zeros(3)
    d = np.zeros(3)
    lib().oracle_primary_ray(_ptr(cam), scene.eye_sep if eye_sep is None else eye_sep,
                             scene.convergence if convergence is None else convergence,
                             scene.W if W is None else W, scene.H if H is None else H,
                             eye, i, j, _ptr(o), _ptr(d))
    return o, d
