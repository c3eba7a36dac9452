"""Seeded synthetic scenes for the stereo ray tracer.

This module only *draws* scenes: primitive positions, sizes, colours,
lights and the stereo camera. It holds none of the tracing arithmetic and
is the one module that both the CUDA path (through the C-ABI) and the CPU
oracle consume, so both sides always see byte-identical inputs.

The paper (Sec. 4) studies scenes of a few polyhedra lit by one light and
prints no scene data, so every scene here is synthetic:

* ``config_small``  - 8 random spheres on a ground plane, one light,
  320x240 per eye, reflection depth 3 (the small plain-method case).
* ``config_blobs``  - 200 displaced icospheres (subdivided 3x, 256,000
  triangles) and 1,000 spheres in a 100^3 box, 4 lights, 30 % mirrors,
  1920x1080 per eye, reflection depth 5 (the plain method at scale).
  ``n_blobs``/``n_spheres``/``W``/``H`` scale it down for parity tests with
  the same distributions.
* ``config_polyhedra`` - the Sec. 4 / Figure 6 scene: two cubes (8 vertices,
  12 triangles), two icosahedra (12 vertices, 20 triangles) and one
  triangulated dodecahedron (20 vertices, 36 triangles) with one light.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) in its counter form: draw k
(k = 0, 1, ...) of a stream seeded with s is mix(s + (k+1)*0x9E3779B97F4A7C15).
U[0,1) = (x >> 11) * 2^-53. A standard normal takes two uniforms u1, u2
(Box-Muller): sqrt(-2 ln(1-u1)) * cos(2 pi u2). The draw order of every
generator is stated in its docstring and never changes.

Struct dtypes mirror the C-ABI structs of ``include/rt_stereo.h`` byte for
byte (little-endian, no padding).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SPHERE_DT = np.dtype([("center", "<f4", (3,)), ("radius", "<f4"), ("material", "<u4")])
TRIANGLE_DT = np.dtype([("v0", "<f4", (3,)), ("v1", "<f4", (3,)), ("v2", "<f4", (3,)),
                        ("material", "<u4")])
MATERIAL_DT = np.dtype([("albedo", "<f4", (3,)), ("reflectivity", "<f4")])
LIGHT_DT = np.dtype([("position", "<f4", (3,)), ("intensity", "<f4")])
CAMERA_DT = np.dtype([("eye", "<f4", (3,)), ("forward", "<f4", (3,)), ("up", "<f4", (3,)),
                      ("vfov_deg", "<f4")])

assert SPHERE_DT.itemsize == 20 and TRIANGLE_DT.itemsize == 40
assert MATERIAL_DT.itemsize == 16 and LIGHT_DT.itemsize == 16 and CAMERA_DT.itemsize == 40

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15
_MIX1 = 0xBF58476D1CE4E5B9
_MIX2 = 0x94D049BB133111EB


class SplitMix64:
    """Counter-form SplitMix64 stream; ``state`` advances by GAMMA per draw."""

    def __init__(self, seed: int):
        self.state = int(seed) & _MASK

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + k * np.uint64(_GAMMA)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(_MIX1)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(_MIX2)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * _GAMMA) & _MASK
        return z

    def uniform(self, n: int) -> np.ndarray:
        """n draws of U[0,1) as float64, 53 random bits each."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        """n standard normals; each consumes two consecutive uniforms."""
        u = self.uniform(2 * n).reshape(n, 2)
        return np.sqrt(-2.0 * np.log1p(-u[:, 0])) * np.cos(2.0 * math.pi * u[:, 1])


@dataclasses.dataclass
class Scene:
    """A stereo rendering request: geometry, materials, lights and camera."""

    name: str
    spheres: np.ndarray      # SPHERE_DT
    triangles: np.ndarray    # TRIANGLE_DT
    materials: np.ndarray    # MATERIAL_DT
    lights: np.ndarray       # LIGHT_DT
    camera: np.ndarray       # CAMERA_DT, shape ()
    eye_sep: float
    convergence: float
    W: int
    H: int
    max_depth: int

    @property
    def n_prims(self) -> int:
        return len(self.spheres) + len(self.triangles)

    def with_view(self, **kw) -> "Scene":
        return dataclasses.replace(self, **kw)


def make_camera(eye, forward, up, vfov_deg) -> np.ndarray:
    cam = np.zeros((), CAMERA_DT)
    cam["eye"] = eye
    cam["forward"] = forward
    cam["up"] = up
    cam["vfov_deg"] = vfov_deg
    return cam


def _tri_array(v: np.ndarray, faces: np.ndarray, material) -> np.ndarray:
    t = np.zeros(len(faces), TRIANGLE_DT)
    t["v0"] = v[faces[:, 0]]
    t["v1"] = v[faces[:, 1]]
    t["v2"] = v[faces[:, 2]]
    t["material"] = material
    return t


def ground_quad(half: float, material: int) -> np.ndarray:
    """The plane y = 0 as two triangles spanning x, z in [-half, half]."""
    v = np.array([[-half, 0, -half], [half, 0, -half], [half, 0, half], [-half, 0, half]],
                 np.float64)
    return _tri_array(v, np.array([[0, 1, 2], [0, 2, 3]]), material)


def config_small(seed: int = 1, W: int = 320, H: int = 240, max_depth: int = 3,
                 n_spheres: int = 8) -> Scene:
    """8 random spheres on a ground plane (the small plain-method case).

    Draw order, per sphere: centre x, y, z; radius; albedo r, g, b;
    reflectivity coin (u < 0.5 -> 0.0, else 0.5). Centres are uniform in
    [-5,5] x [0,3] x [-15,-5], radii in [0.3, 1.2). Material i belongs to
    sphere i; the last material is the ground (albedo 0.8, not reflective).
    The ground plane y = 0 is a quad spanning x, z in [-1000, 1000]; one white
    point light of intensity 1 sits at (0, 10, 0). The centre eye is at
    (0, 2, 0) looking down -z with 60 deg vertical field of view; the
    convergence plane z = -10 lies 10 units ahead; eye separation 0.065.
    """
    rng = SplitMix64(seed)
    u = rng.uniform(8 * n_spheres).reshape(n_spheres, 8)
    sp = np.zeros(n_spheres, SPHERE_DT)
    sp["center"][:, 0] = -5.0 + 10.0 * u[:, 0]
    sp["center"][:, 1] = 0.0 + 3.0 * u[:, 1]
    sp["center"][:, 2] = -15.0 + 10.0 * u[:, 2]
    sp["radius"] = 0.3 + 0.9 * u[:, 3]
    sp["material"] = np.arange(n_spheres)
    mats = np.zeros(n_spheres + 1, MATERIAL_DT)
    mats["albedo"][:n_spheres] = u[:, 4:7]
    mats["reflectivity"][:n_spheres] = np.where(u[:, 7] < 0.5, 0.0, 0.5)
    mats["albedo"][n_spheres] = 0.8
    tris = ground_quad(1000.0, n_spheres)
    lights = np.zeros(1, LIGHT_DT)
    lights["position"] = (0.0, 10.0, 0.0)
    lights["intensity"] = 1.0
    cam = make_camera((0, 2, 0), (0, 0, -1), (0, 1, 0), 60.0)
    return Scene(f"small-seed{seed}", sp, tris, mats, lights, cam, 0.065, 10.0, W, H, max_depth)


# ---------------------------------------------------------------- polyhedra
_PHI = (1.0 + math.sqrt(5.0)) / 2.0


def _faces_by_edge_length(v: np.ndarray, edge: float) -> np.ndarray:
    """All vertex triples whose three pairwise distances equal ``edge``."""
    n = len(v)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=-1)
    adj = np.abs(d - edge) < 1e-9
    out = []
    for i in range(n):
        for j in range(i + 1, n):
            if not adj[i, j]:
                continue
            for k in range(j + 1, n):
                if adj[i, k] and adj[j, k]:
                    out.append((i, j, k))
    return np.array(out, np.int64)


def icosahedron() -> tuple[np.ndarray, np.ndarray]:
    """12 vertices (cyclic permutations of (0, +-1, +-phi)), 20 faces."""
    v = []
    for a in (-1.0, 1.0):
        for b in (-_PHI, _PHI):
            v += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    v = np.array(v)
    return v, _faces_by_edge_length(v, 2.0)


def cube() -> tuple[np.ndarray, np.ndarray]:
    """8 vertices, 12 triangles (each square face split along a diagonal)."""
    v = np.array([[x, y, z] for x in (-1.0, 1.0) for y in (-1.0, 1.0) for z in (-1.0, 1.0)])
    faces = []
    for axis in range(3):
        for s in (-1.0, 1.0):
            idx = [i for i in range(8) if v[i, axis] == s]
            a, b, c, d = _order_polygon(v, idx)
            faces += [(a, b, c), (a, c, d)]
    return v, np.array(faces, np.int64)


def _order_polygon(v: np.ndarray, idx) -> list[int]:
    """Order the coplanar vertices ``idx`` by angle around their centroid."""
    p = v[idx]
    c = p.mean(axis=0)
    n = c / np.linalg.norm(c)
    e1 = p[0] - c
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    ang = [math.atan2(np.dot(q - c, e2), np.dot(q - c, e1)) for q in p]
    return [idx[i] for i in np.argsort(ang)]


def dodecahedron() -> tuple[np.ndarray, np.ndarray]:
    """20 vertices, 12 pentagons fan-split into 36 triangles.

    Each pentagon is the set of the 5 vertices nearest to the direction of
    one icosahedron vertex (the two solids are dual).
    """
    ip = 1.0 / _PHI
    v = [[x, y, z] for x in (-1.0, 1.0) for y in (-1.0, 1.0) for z in (-1.0, 1.0)]
    for a in (-1.0, 1.0):
        for b in (-1.0, 1.0):
            v += [[0.0, a * ip, b * _PHI], [a * ip, b * _PHI, 0.0], [a * _PHI, 0.0, b * ip]]
    v = np.array(v)
    iv, _ = icosahedron()
    faces = []
    # the dual icosahedron of this dodecahedron has its vertices at the
    # cyclic permutations of (0, +-phi, +-1): swap y and z of ours
    for dvec in iv[:, [0, 2, 1]]:
        idx = list(np.argsort(-(v @ dvec))[:5])
        a, b, c, d, e = _order_polygon(v, idx)
        faces += [(a, b, c), (a, c, d), (a, d, e)]
    return v, np.array(faces, np.int64)


def icosphere(subdiv: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit icosphere: each subdivision splits a face into 4 at edge midpoints
    (projected back onto the sphere). 10*4^s + 2 vertices, 20*4^s faces."""
    v, f = icosahedron()
    verts = [tuple(x / np.linalg.norm(x)) for x in v]
    faces = [tuple(t) for t in f]
    for _ in range(subdiv):
        cache: dict[tuple[int, int], int] = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = np.add(verts[a], verts[b]) * 0.5
                verts.append(tuple(m / np.linalg.norm(m)))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts), np.array(faces, np.int64)


def splitmix64_at(seed: int, counter: np.ndarray) -> np.ndarray:
    """Draw number ``counter`` (0-based) of the SplitMix64 stream seeded with
    ``seed``, for an array of counters (random access into the stream)."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(int(seed) & _MASK) + (c + np.uint64(1)) * np.uint64(_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_MIX2)
        z = z ^ (z >> np.uint64(31))
    return z


def value_noise(seed: int, x: np.ndarray, z: np.ndarray) -> np.ndarray:
    """2-D value noise in [-1, 1]: lattice values 2U - 1 with U = draw
    (ix mod 2^20) * 2^20 + (iz mod 2^20) of SplitMix64(seed), blended
    bilinearly with smoothstep weights 3t^2 - 2t^3."""
    fx, fz = np.floor(x), np.floor(z)
    tx, tz = x - fx, z - fz
    ix, iz = fx.astype(np.int64), fz.astype(np.int64)

    def lat(a, b):
        k = ((a & 0xFFFFF) << 20) | (b & 0xFFFFF)
        u = (splitmix64_at(seed, k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return 2.0 * u - 1.0

    sx, sz = tx * tx * (3.0 - 2.0 * tx), tz * tz * (3.0 - 2.0 * tz)
    a = lat(ix, iz) + (lat(ix + 1, iz) - lat(ix, iz)) * sx
    b = lat(ix, iz + 1) + (lat(ix + 1, iz + 1) - lat(ix, iz + 1)) * sx
    return a + (b - a) * sz


def fbm(seed: int, x: np.ndarray, z: np.ndarray, octaves: int = 6, wavelength: float = 250.0):
    """Fractional Brownian motion: sum over octaves o of 0.5^o times value
    noise (seed + o) at frequency 2^o / wavelength."""
    h = np.zeros(np.broadcast(x, z).shape)
    for o in range(octaves):
        f = (2.0 ** o) / wavelength
        h += (0.5 ** o) * value_noise(seed + o, x * f, z * f)
    return h


def config_terrain(seed: int = 5, n_grid: int = 2236, n_spheres: int = 10000, n_lights: int = 8,
                   W: int = 3840, H: int = 2160, max_depth: int = 4, size: float = 1000.0,
                   amplitude: float = 60.0) -> Scene:
    """Procedural terrain: an n_grid x n_grid height grid over [-size, size]^2
    (2 (n_grid-1)^2 triangles; 9,990,450 for 2236), height amplitude * fbm
    (6 octaves of value noise, base wavelength size/4, seed), plus n_spheres
    spheres floating over it and n_lights point lights.

    Cell (i, j) with corners v00 = (i, j), v10 = (i+1, j), v01 = (i, j+1),
    v11 = (i+1, j+1) gives triangles (v00, v10, v11) and (v00, v11, v01);
    material 0 (albedo (0.45, 0.5, 0.35), matte) is the terrain. Spheres
    draw from SplitMix64(seed + 100), 8 uniforms each in this order: x, z
    (U[-0.9 size, 0.9 size]), radius U[0.5, 4), lift U[0, 20) above the
    terrain (centre y = height(x, z) + radius + lift), albedo r, g, b, mirror
    coin (u < 0.3 -> reflectivity 0.7); sphere s has material 1 + s. Lights
    draw x, z (U[-size, size]) and sit at y = 400 with intensity 1/n_lights.
    The camera is frame 0 of ``terrain_cameras``.
    """
    g = np.linspace(-size, size, n_grid)
    X, Z = np.meshgrid(g, g, indexing="ij")
    Y = amplitude * fbm(seed, X, Z, wavelength=size / 4.0)
    V = np.stack([X, Y, Z], -1).astype(np.float32)
    i, j = np.meshgrid(np.arange(n_grid - 1), np.arange(n_grid - 1), indexing="ij")
    i, j = i.ravel(), j.ravel()
    v00, v10, v01, v11 = V[i, j], V[i + 1, j], V[i, j + 1], V[i + 1, j + 1]
    tris = np.zeros(2 * len(i), TRIANGLE_DT)
    tris["v0"][0::2], tris["v1"][0::2], tris["v2"][0::2] = v00, v10, v11
    tris["v0"][1::2], tris["v1"][1::2], tris["v2"][1::2] = v00, v11, v01
    tris["material"] = 0
    mats = np.zeros(1 + n_spheres, MATERIAL_DT)
    mats["albedo"][0] = (0.45, 0.5, 0.35)
    sp = np.zeros(n_spheres, SPHERE_DT)
    if n_spheres:
        u = SplitMix64(seed + 100).uniform(8 * n_spheres).reshape(n_spheres, 8)
        x = -0.9 * size + 1.8 * size * u[:, 0]
        z = -0.9 * size + 1.8 * size * u[:, 1]
        r = 0.5 + 3.5 * u[:, 2]
        y = amplitude * fbm(seed, x, z, wavelength=size / 4.0) + r + 20.0 * u[:, 3]
        sp["center"] = np.stack([x, y, z], -1)
        sp["radius"] = r
        sp["material"] = 1 + np.arange(n_spheres)
        mats["albedo"][1:] = u[:, 4:7]
        mats["reflectivity"][1:] = np.where(u[:, 7] < 0.3, 0.7, 0.0)
    lights = np.zeros(n_lights, LIGHT_DT)
    u = SplitMix64(seed + 200).uniform(2 * n_lights).reshape(n_lights, 2)
    lights["position"] = np.stack([-size + 2 * size * u[:, 0], np.full(n_lights, 400.0),
                                   -size + 2 * size * u[:, 1]], -1)
    lights["intensity"] = 1.0 / n_lights
    cams = terrain_cameras(seed, 1, size=size, amplitude=amplitude)
    return Scene(name=f"terrain-{seed}", spheres=sp, triangles=tris, materials=mats, lights=lights,
                 camera=cams[0], eye_sep=0.065, convergence=60.0, W=W, H=H, max_depth=max_depth)


def terrain_cameras(seed: int = 5, n_frames: int = 120, n_keys: int = 8, size: float = 1000.0,
                    amplitude: float = 60.0, frames_per_loop: int = 120) -> np.ndarray:
    """Cameras of a flight over the terrain: a closed uniform Catmull-Rom
    spline through n_keys control points drawn from SplitMix64(seed + 300)
    (x, z in U[-0.6 size, 0.6 size], y = terrain height + 30 + U[0, 20), 3
    uniforms per key in that order). Frame f sits at spline parameter
    n_keys * f / frames_per_loop, raised where needed to 20 above the terrain;
    it looks along the spline tangent tilted down by 0.3 (before
    normalisation), up = +y, 60 degree field of view."""
    u = SplitMix64(seed + 300).uniform(3 * n_keys).reshape(n_keys, 3)
    kx = -0.6 * size + 1.2 * size * u[:, 0]
    kz = -0.6 * size + 1.2 * size * u[:, 1]
    ky = amplitude * fbm(seed, kx, kz, wavelength=size / 4.0) + 30.0 + 20.0 * u[:, 2]
    K = np.stack([kx, ky, kz], -1)

    def spline(t):
        k = int(np.floor(t)) % n_keys
        s_ = t - np.floor(t)
        p0, p1, p2, p3 = K[(k - 1) % n_keys], K[k], K[(k + 1) % n_keys], K[(k + 2) % n_keys]
        return 0.5 * ((2 * p1) + (-p0 + p2) * s_ + (2 * p0 - 5 * p1 + 4 * p2 - p3) * s_ ** 2
                      + (-p0 + 3 * p1 - 3 * p2 + p3) * s_ ** 3)

    cams = np.zeros(n_frames, CAMERA_DT)
    for f in range(n_frames):
        t = n_keys * f / frames_per_loop
        e = spline(t)
        d = spline(t + 1e-3) - e
        ground = amplitude * fbm(seed, np.array([e[0]]), np.array([e[2]]), wavelength=size / 4.0)[0]
        e[1] = max(e[1], ground + 20.0)
        d = d / np.linalg.norm(d)
        d[1] -= 0.3
        cams["eye"][f] = e
        cams["forward"][f] = d / np.linalg.norm(d)
        cams["up"][f] = (0.0, 1.0, 0.0)
        cams["vfov_deg"][f] = 60.0
    return cams


BATCH_RESOLUTIONS = ((640, 360), (1280, 720), (1920, 1080), (3840, 2160))


def config_batch(seed: int = 3, n_scenes: int = 16, n_requests: int = 64):
    """The batched workload: n_requests stereo requests over n_scenes blob
    scenes whose triangle counts are log-spaced from 1e3 to 2e6.

    Scene k has n_blobs = max(1, round(1e3 * 2000^(k/(n_scenes-1)) / 1280))
    displaced icospheres (1,280 triangles each) and 5 spheres per blob, built
    by ``config_blobs`` with seed 100*seed + k, 4 lights, and a box scaled by
    (n_blobs/200)^(1/3) so the density matches the 200-blob scene. Request i
    draws (from SplitMix64(seed), three uniforms per request in this order)
    its scene index floor(16 u), its per-eye resolution
    BATCH_RESOLUTIONS[floor(4 u)] and its reflection depth 2 + floor(5 u).
    Returns (scenes, [(scene index, W, H, max_depth), ...]).
    """
    scenes = []
    for k in range(n_scenes):
        ntri = 1e3 * 2000.0 ** (k / max(1, n_scenes - 1))
        nb = max(1, int(round(ntri / 1280.0)))
        scenes.append(config_blobs(100 * seed + k, n_blobs=nb, n_spheres=5 * nb,
                                   box=50.0 * (nb / 200.0) ** (1.0 / 3.0)))
    u = SplitMix64(seed).uniform(3 * n_requests).reshape(n_requests, 3)
    reqs = []
    for i in range(n_requests):
        si = min(n_scenes - 1, int(u[i, 0] * n_scenes))
        W, H = BATCH_RESOLUTIONS[min(3, int(u[i, 1] * 4))]
        reqs.append((si, W, H, 2 + min(4, int(u[i, 2] * 5))))
    return scenes, reqs


def config_polyhedra(n_objects: int = 5, n_lights: int = 1, W: int = 320, H: int = 240,
                     max_depth: int = 3, ground: bool = False) -> Scene:
    """The Sec. 4 test scenes (Figures 3-7): up to 6 polyhedra and 1-8 lights.

    Objects in order: cube, cube, icosahedron, icosahedron, dodecahedron,
    icosphere(1) (the sixth, "different complexity" object of Figure 7).
    With 5 objects this is the Figure 6 scene: two objects of 8 vertices / 12
    polygons, two of 12 vertices / 20 polygons and one of 20 vertices / 36
    polygons. Placement, colours and lights are fixed (no randomness): the
    paper prints none. Object k sits at x = -5 + 2.5k, y = 1, z = -8 (sixth
    at x = 0, y = 3.2, z = -10) with circumradius ~1.
    """
    shapes = [cube(), cube(), icosahedron(), icosahedron(), dodecahedron(), icosphere(1)]
    cols = [(0.9, 0.2, 0.2), (0.2, 0.9, 0.2), (0.2, 0.3, 0.9), (0.9, 0.9, 0.2),
            (0.8, 0.4, 0.9), (0.7, 0.7, 0.7)]
    refl = [0.0, 0.5, 0.0, 0.5, 0.0, 0.5]
    tris = []
    mats = np.zeros(n_objects + 1, MATERIAL_DT)
    for k in range(n_objects):
        v, f = shapes[k]
        v = v / np.max(np.linalg.norm(v, axis=1))
        pos = (-5.0 + 2.5 * k, 1.0, -8.0) if k < 5 else (0.0, 3.2, -10.0)
        tris.append(_tri_array(v + np.array(pos), f, k))
        mats["albedo"][k] = cols[k]
        mats["reflectivity"][k] = refl[k]
    mats["albedo"][n_objects] = 0.8
    if ground:
        tris.append(ground_quad(1000.0, n_objects))
    tris = np.concatenate(tris) if tris else np.zeros(0, TRIANGLE_DT)
    lights = np.zeros(n_lights, LIGHT_DT)
    for l in range(n_lights):
        a = 2.0 * math.pi * l / max(n_lights, 1)
        lights["position"][l] = (8.0 * math.sin(a), 10.0, -8.0 + 8.0 * math.cos(a))
        lights["intensity"][l] = 1.0 / n_lights
    cam = make_camera((0, 2, 0), (0, 0, -1), (0, 1, 0), 60.0)
    return Scene(f"polyhedra-{n_objects}obj-{n_lights}l", np.zeros(0, SPHERE_DT), tris, mats,
                 lights, cam, 0.065, 10.0, W, H, max_depth)


def config_blobs(seed: int = 2, n_blobs: int = 200, n_spheres: int = 1000, n_lights: int = 4,
                 subdiv: int = 3, W: int = 1920, H: int = 1080, max_depth: int = 5,
                 box: float = 50.0) -> Scene:
    """Displaced icosphere blobs and spheres in a (2*box)^3 cube.

    Draw order: for each blob: centre x, y, z (U[-box, box]); radius
    U[0.5, 3); albedo r, g, b; mirror coin (u < 0.3 -> reflectivity 0.7,
    else 0); then one standard normal per icosphere vertex, in vertex order
    (each vertex moves along its normal by N(0,1) * 0.1 * radius). Then for
    each sphere: centre x, y, z; radius U[0.05, 0.5); albedo r, g, b; mirror
    coin. Then for each light: x, z (U[-box, box]); lights sit at
    y = 1.2 * box with intensity 1/L. Material b belongs to blob b, material
    n_blobs + s to sphere s. The centre eye is at (0, 0, 1.8 * box) looking
    down -z, 60 deg vertical field of view, converging on the plane z = 0,
    eye separation 0.065.
    """
    rng = SplitMix64(seed)
    unit_v, faces = icosphere(subdiv)
    nv = len(unit_v)
    tris = []
    mats = np.zeros(n_blobs + n_spheres, MATERIAL_DT)
    for b in range(n_blobs):
        u = rng.uniform(8)
        c = -box + 2.0 * box * u[0:3]
        r = 0.5 + 2.5 * u[3]
        mats["albedo"][b] = u[4:7]
        mats["reflectivity"][b] = 0.7 if u[7] < 0.3 else 0.0
        z = rng.normal(nv)
        v = c + unit_v * (r * (1.0 + 0.1 * z))[:, None]
        tris.append(_tri_array(v, faces, b))
    tris = np.concatenate(tris) if tris else np.zeros(0, TRIANGLE_DT)
    sp = np.zeros(n_spheres, SPHERE_DT)
    if n_spheres:
        u = rng.uniform(8 * n_spheres).reshape(n_spheres, 8)
        sp["center"] = -box + 2.0 * box * u[:, 0:3]
        sp["radius"] = 0.05 + 0.45 * u[:, 3]
        sp["material"] = n_blobs + np.arange(n_spheres)
        mats["albedo"][n_blobs:] = u[:, 4:7]
        mats["reflectivity"][n_blobs:] = np.where(u[:, 7] < 0.3, 0.7, 0.0)
    lights = np.zeros(n_lights, LIGHT_DT)
    u = rng.uniform(2 * n_lights).reshape(n_lights, 2)
    lights["position"][:, 0] = -box + 2.0 * box * u[:, 0]
    lights["position"][:, 1] = 1.2 * box
    lights["position"][:, 2] = -box + 2.0 * box * u[:, 1]
    lights["intensity"] = 1.0 / n_lights
    cam = make_camera((0, 0, 1.8 * box), (0, 0, -1), (0, 1, 0), 60.0)
    return Scene(f"blobs-seed{seed}-{n_blobs}b{n_spheres}s", sp, tris, mats, lights, cam,
                 0.065, 1.8 * box, W, H, max_depth)


def describe(scene: Scene) -> dict:
    return {"name": scene.name, "spheres": int(len(scene.spheres)),
            "triangles": int(len(scene.triangles)), "lights": int(len(scene.lights)),
            "W": scene.W, "H": scene.H, "max_depth": scene.max_depth,
            "eye_sep": scene.eye_sep, "convergence": scene.convergence}


# ----------------------------------------------------- reprojection inputs
def gbuffer_synthetic(seed: int, W: int, H: int, miss_frac: float = 0.2,
                      z_lo: float = 2.0, z_hi: float = 60.0):
    """A random left-eye G-buffer (test input for the forward warp).

    Draw order per pixel (row-major): miss coin, depth u (log-uniform in
    [z_lo, z_hi)), normal x, y, z (uniform in [-1,1], then normalised), id u
    (ids 0..999), r, g, b. Misses get depth +inf and id 0xFFFFFFFF. The
    hit surface's reflectivity is (0, 0.5, 0.7)[id % 3] (0 on a miss).
    Returns float32 depth (P), normal (P,3), rgb (P,3), uint32 ids (P) and
    float32 reflectivity (P).
    """
    u = SplitMix64(seed).uniform(W * H * 9).reshape(W * H, 9)
    miss = u[:, 0] < miss_frac
    depth = (z_lo * (z_hi / z_lo) ** u[:, 1]).astype(np.float32)
    depth[miss] = np.inf
    n = 2.0 * u[:, 2:5] - 1.0
    n /= np.maximum(np.linalg.norm(n, axis=1, keepdims=True), 1e-12)
    ids = np.minimum((u[:, 5] * 1000).astype(np.uint32), 999).astype(np.uint32)
    ids[miss] = 0xFFFFFFFF
    refl = np.array([0.0, 0.5, 0.7], np.float32)[ids % 3]
    refl[miss] = 0.0
    return depth, n.astype(np.float32), ids, u[:, 6:9].astype(np.float32), refl


NET_LAYERS = ((10, 32), (32, 32), (32, 32), (32, 1))
NET_PARAMS = sum(co * ci * 9 + co for ci, co in NET_LAYERS)


def net_params_he(seed: int) -> np.ndarray:
    """He-normal initial weights (N(0, 2/(9 Cin))), zero biases, in the
    parameter order W1, b1, W2, b2, W3, b3, W4, b4 (W as [Cout][Cin][3][3]).
    Draw order: the weights of layer 1..4, each in that layout's order."""
    rng = SplitMix64(seed)
    out = []
    for ci, co in NET_LAYERS:
        w = rng.normal(co * ci * 9) * np.sqrt(2.0 / (9 * ci))
        out += [w, np.zeros(co)]
    p = np.concatenate(out).astype(np.float32)
    assert p.size == NET_PARAMS
    return p


def bf16_features_synthetic(seed: int, W: int, H: int) -> np.ndarray:
    """Random network inputs already representable in BF16: (P, 16) float32,
    channels 0-9 uniform in [-1, 1) rounded to 8 significant bits, 10-15 zero."""
    c = NET_LAYERS[0][0]
    u = SplitMix64(seed).uniform(W * H * c).reshape(W * H, c) * 2.0 - 1.0
    f = np.zeros((W * H, 16), np.float32)
    m, e = np.frexp(u)
    f[:, :c] = np.ldexp(np.round(m * 256.0) / 256.0, e)
    return f
