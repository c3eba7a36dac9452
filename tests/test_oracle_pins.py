"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Nothing here compares the oracle with itself: every expected value is a
closed form worked out for the scene at hand, an exact symmetry, a second
independent algorithm, or a count the paper prints.

Readings of the paper used below (it specifies no shading model): ambient
k_a = 0.1, white point lights without distance falloff, background
(0.2, 0.3, 0.5), colour = (1-r) local + r reflected, reflected term 0 at the
maximum depth, secondary origins offset by 1e-4 max(1, |p|_inf) along the
normal facing the incoming ray.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1702_01530_gb300 import scenegen as sg
from tests.scenes_util import quad, quad_xz, scene

KA = 0.1
BG = np.array([0.2, 0.3, 0.5])
MISS = 0xFFFFFFFF


# ------------------------------------------------------------------ T1 sphere
def _sphere_scene(light_pos, intensity=1.0, albedo=(0.4, 0.6, 0.8)):
    return scene(spheres=[((0, 0, -10), 1.0, 0)], mats=[(*albedo, 0.0)],
                 lights=[(light_pos, intensity)], W=33, H=33)


def test_sphere_closed_form_hit_and_depth():
    s = _sphere_scene((0, 0, 1))
    osc = oracle.OracleScene(s)
    t, pid, tie = osc.closest([0, 0, 0], [0, 0, -1])
    assert (t, pid, tie) == (9.0, 0, False)              # d - r
    t, pid, _ = osc.closest([0, 0.5, 0], [0, 0, -1])
    assert abs(t - (10.0 - math.sqrt(1 - 0.25))) < 1e-12
    t, pid, _ = osc.closest([0, 0, -10], [0, 1, 0])      # from the centre: far root
    assert abs(t - 1.0) < 1e-15
    t, pid, _ = osc.closest([0, 0, 0], [0, 0, 1])        # pointing away: miss
    assert pid == MISS and t == math.inf
    _, pid, tie = osc.closest([0, 1.0, 0], [0, 0, -1])   # tangent ray: a near tie
    assert tie


def test_sphere_closed_form_shading():
    # light on the surface normal of the hit point (0,0,-9): n.l = 1
    alb = np.array([0.4, 0.6, 0.8])
    r = oracle.render(_sphere_scene((0, 0, 1), intensity=0.7))
    c = 16
    assert r["hit_id"][0, c, c] == 0 and r["depth"][0, c, c] == 9.0
    assert np.allclose(r["rgb"][0, c, c], alb * (KA + 0.7), atol=1e-12)
    assert np.array_equal(r["rgb"][0, 0, 0], BG) and r["hit_id"][0, 0, 0] == MISS
    # light at 60 deg from the normal, seen from the offset origin: n.l = 0.5
    eps = 1e-4 * 9.0
    o2 = np.array([0, 0, -9.0 + eps])
    lp = o2 + 10.0 * np.array([0, math.sin(math.pi / 3), math.cos(math.pi / 3)])
    r = oracle.render(_sphere_scene(tuple(lp)))
    lp32 = lp.astype(np.float32).astype(np.float64)
    ndl = (lp32 - o2)[2] / np.linalg.norm(lp32 - o2)
    assert abs(ndl - 0.5) < 1e-6
    assert np.allclose(r["rgb"][0, c, c], alb * (KA + ndl), atol=1e-12)
    # light behind the surface: no shadow ray, ambient only
    r = oracle.render(_sphere_scene((0, 0, -30)))
    assert np.allclose(r["rgb"][0, c, c], alb * KA, atol=1e-15)


# ---------------------------------------------------------------- T2 triangle
def test_triangle_moller_trumbore_closed_forms():
    s = scene(tris=[((0, 0, -5), (2, 0, -5), (0, 2, -5), 0)])
    osc = oracle.OracleScene(s)
    assert osc.closest([0.5, 0.5, 0], [0, 0, -1]) == (5.0, 0, False)
    t, pid, tie = osc.closest([1.0, 1.0, 0], [0, 0, -1])     # on the edge u + v = 1
    assert pid == 0 and t == 5.0 and tie                      # inclusive, flagged
    assert osc.closest([1.2, 0.5, 0], [0, 0, -1])[1] == 0     # u + v = 0.85
    assert osc.closest([1.2, 0.9, 0], [0, 0, -1])[1] == MISS  # u + v = 1.05
    t, pid, tie = osc.closest([-1e-12, 0.5, 0], [0, 0, -1])   # just outside u = 0
    assert pid == MISS and tie
    t, pid, _ = osc.closest([0.5, 0.5, -10], [0, 0, 1])       # back face: two-sided
    assert (t, pid) == (5.0, 0)
    t, pid, tie = osc.closest([0.5, 0.5, -5], [1, 0, 0])      # in the plane
    assert pid == MISS and tie
    d = np.array([0.5, 0.5, -5.0])
    t, pid, _ = osc.closest([0, 0, 0], d / np.linalg.norm(d))
    assert pid == 0 and abs(t - np.linalg.norm(d)) < 1e-12
    t, pid, _ = osc.closest([0, 0, 0], d)                     # unnormalised direction
    assert abs(t - 1.0) < 1e-15


def test_closest_hit_tie_break_lower_id():
    # two coincident triangles: equal t -> the lower primitive id wins
    tri = ((-1, -1, -4), (1, -1, -4), (0, 1, -4))
    s = scene(spheres=[((0, 0, -20), 1.0, 0)], tris=[(*tri, 0), (*tri, 0)])
    t, pid, tie = oracle.OracleScene(s).closest([0, 0, 0], [0, 0, -1])
    assert (t, pid, tie) == (4.0, 1, True)    # ids: sphere 0, triangles 1, 2


# -------------------------------------------------------- T3 stereo invariants
def test_zero_separation_gives_identical_eyes():
    s = sg.config_small(1, W=96, H=72).with_view(eye_sep=0.0)
    r = oracle.render(s)
    assert np.array_equal(r["rgb"][0], r["rgb"][1])
    assert np.array_equal(r["hit_id"][0], r["hit_id"][1])


def test_mirror_symmetric_scene_gives_mirrored_eyes():
    # a scene symmetric under x -> -x: the left eye (at -s/2) sees the mirror
    # image of what the right eye (at +s/2) sees
    mats = [(0.8, 0.3, 0.3, 0.5), (0.3, 0.8, 0.3, 0.0), (0.7, 0.7, 0.7, 0.0)]
    s = scene(spheres=[((-2, 1, -8), 1.0, 0), ((2, 1, -8), 1.0, 0), ((0, 0.6, -6), 0.6, 1)],
              tris=quad_xz(-50, 50, -50, 50, 0.0, 2), mats=mats,
              lights=[((0, 10, -5), 1.0)], eye=(0, 1.5, 0), W=64, H=48,
              eye_sep=0.4, convergence=7.0, max_depth=3)
    r = oracle.render(s)
    L, R = r["rgb"][0], r["rgb"][1][:, ::-1]
    ok = (r["flags"][0] == 0) & (r["flags"][1][:, ::-1] == 0)
    assert ok.mean() > 0.95
    assert np.abs(L - R)[ok].max() < 1e-9
    assert not np.allclose(r["rgb"][0], r["rgb"][1])   # the eyes do differ


def test_image_orientation_row0_top_and_right_is_plus_x():
    # camera at the origin looking down -z with +y up: a sphere above the
    # view axis lands in the top rows, one at +x in the right half
    for centre, where in (((0, 2.5, -10), "top"), ((3.5, 0, -10), "right")):
        s = scene(spheres=[(centre, 1.0, 0)], W=40, H=30)
        hit = oracle.render(s)["hit_id"][0] != MISS
        rows, cols = np.nonzero(hit)
        assert len(rows) > 10
        if where == "top":
            assert rows.max() < 15 and abs(cols.mean() - 19.5) < 1
        else:
            assert cols.min() > 20 and abs(rows.mean() - 14.5) < 1


# ------------------------------------------------------------ T4 disparity
def _disparity_scene(W=200, H=480, s=1.0, zc=8.0, z=4.0, tiles=True):
    vfov = math.degrees(2 * math.atan(0.5))          # tan(vfov/2) = 1/2: f_px = H
    tris = []
    if tiles:
        k = 0
        for a in range(-6, 6):
            for b in range(-6, 6):
                tris += quad(0.5 * a, 0.5 * (a + 1), 0.5 * b, 0.5 * (b + 1), -z, 0)
                k += 1
    return scene(tris=tris, W=W, H=H, vfov=vfov, eye_sep=s, convergence=zc,
                 lights=[((0, 0, 5), 1.0)], max_depth=0)


def test_disparity_closed_form_ray_level():
    W, H, s, zc, z = 200, 480, 1.0, 8.0, 4.0
    sc = _disparity_scene(W, H, s, zc, z, tiles=False)
    f_px = (H / 2) / math.tan(math.radians(float(np.float32(sc.camera["vfov_deg"]))) / 2)
    D = f_px * s * (1 / z - 1 / zc)
    assert abs(D - 60.0) < 1e-4                       # x_L - x_R in pixels
    for i, j in [(0, 0), (17, 100), (70, 239), (139, 479)]:
        oR, dR = oracle.primary_ray(sc, +1, i, j)
        oL, dL = oracle.primary_ray(sc, -1, i + 60, j)
        pR = oR + dR * ((-z - oR[2]) / dR[2])
        pL = oL + dL * ((-z - oL[2]) / dL[2])
        assert np.abs(pR - pL).max() < 1e-4           # same point of the plane
        # both eyes' rays through pixel (i, j) meet on the convergence plane
        oL2, dL2 = oracle.primary_ray(sc, -1, i, j)
        qR = oR + dR * ((-zc - oR[2]) / dR[2])
        qL = oL2 + dL2 * ((-zc - oL2[2]) / dL2[2])
        assert np.abs(qR - qL).max() < 1e-12
        assert abs(oR[0] - oL2[0] - s) < 1e-15 and oR[1] == oL2[1]
        assert np.linalg.norm(dR) == pytest.approx(1.0, abs=1e-15)


def test_disparity_closed_form_image_level():
    r = oracle.render(_disparity_scene())
    hL, hR = r["hit_id"][0], r["hit_id"][1]
    fl = (r["flags"][0] | r["flags"][1]) & 1
    hitL, hitR = hL[:, 60:], hR[:, :-60]
    ok = (fl[:, 60:] == 0) & (fl[:, :-60] == 0) & (hitR != MISS)
    assert ok.sum() > 10000
    assert np.array_equal(hitL[ok], hitR[ok])


# --------------------------------------------------------- T5 brute vs BVH
@pytest.mark.parametrize("nb,sub,ns", [(0, 0, 65), (1, 1, 20), (2, 2, 40), (3, 3, 100)])
def test_bvh_equals_brute_force(nb, sub, ns):
    s = sg.config_blobs(seed=7 + nb, n_blobs=nb, n_spheres=ns, subdiv=sub, W=48, H=36,
                        max_depth=3, box=6.0)
    osc = oracle.OracleScene(s)
    a = osc.render(mode=osc.MODE_BRUTE)
    b = osc.render(mode=osc.MODE_BVH)
    assert (a["hit_id"] != MISS).mean() > 0.1
    for k in ("rgb", "hit_id", "depth", "flags", "rays"):
        assert np.array_equal(a[k], b[k]), k
    assert b["work"][0, 0] > 0 and a["work"].sum() == 0


# ------------------------------------------------------------------ T6 LBVH
def _interleave_by_strings(qx, qy, qz):
    bx, by, bz = (format(q, "010b") for q in (qx, qy, qz))
    return int("".join(x + y + z for x, y, z in zip(bx, by, bz)), 2)


def test_morton_interleave():
    assert oracle.morton30(1, 0, 0) == 4
    assert oracle.morton30(0, 1, 0) == 2
    assert oracle.morton30(0, 0, 1) == 1
    assert oracle.morton30(1023, 1023, 1023) == (1 << 30) - 1
    rng = np.random.default_rng(0)
    for qx, qy, qz in rng.integers(0, 1024, size=(200, 3)):
        assert oracle.morton30(int(qx), int(qy), int(qz)) == _interleave_by_strings(qx, qy, qz)


def _spheres_at(xs):
    return scene(spheres=[((float(x), 0.0, 0.0), 0.25, 0) for x in xs])


def test_lbvh_keys_quantisation():
    b = oracle.OracleScene(_spheres_at([0, 1, 2, 3])).lbvh()
    # x in [0,3]: q = floor(x/3*1024) = 0, 341, 682, 1024 -> 1023; y, z extent 0
    expect = sorted((_interleave_by_strings(q, 0, 0) << 32) | i
                    for i, q in enumerate([0, 341, 682, 1023]))
    assert b["keys"].tolist() == expect


def test_lbvh_quantisation_uses_1024_cells():
    # x = 0, 0.5, 1 on [0, 1]: floor(0.5 * 1024) = 512 (a 1023-cell grid would give 511)
    b = oracle.OracleScene(_spheres_at([0, 0.5, 1])).lbvh()
    expect = sorted((_interleave_by_strings(q, 0, 0) << 32) | i for i, q in enumerate([0, 512, 1023]))
    assert b["keys"].tolist() == expect


def test_lbvh_hand_worked_trees():
    b = oracle.OracleScene(_spheres_at([0])).lbvh()
    assert b["left"].size == 0 and b["parent"].tolist() == [-1]
    b = oracle.OracleScene(_spheres_at([0, 1])).lbvh()
    assert b["left"].tolist() == [-1] and b["right"].tolist() == [-2]
    assert b["parent"].tolist() == [-1, 0, 0]
    # x = 0, 1, 1023 on [0, 1023]: q = 0, 1, 1023; the split of [0,2] is after 1
    b = oracle.OracleScene(_spheres_at([0, 1, 1023])).lbvh()
    assert b["left"].tolist() == [1, -1] and b["right"].tolist() == [-3, -2]
    assert b["parent"].tolist() == [-1, 0, 1, 1, 0]
    # 8 coincident centroids: keys are the ids 0..7, a perfect binary tree
    b = oracle.OracleScene(_spheres_at([5.0] * 8)).lbvh()
    assert b["keys"].tolist() == list(range(8))
    assert b["left"].tolist() == [3, ~0, ~2, 1, 5, ~4, ~6]
    assert b["right"].tolist() == [4, ~1, ~3, 2, 6, ~5, ~7]


def _clz64(x):
    return 64 - int(x).bit_length()


def _karras_per_node(keys):
    """Karras (HPG 2012) per-node construction: direction, range, split."""
    n = len(keys)
    keys = [int(k) for k in keys]

    def delta(i, j):
        return -1 if j < 0 or j >= n else _clz64(keys[i] ^ keys[j])

    left, right = [0] * (n - 1), [0] * (n - 1)
    for i in range(n - 1):
        d = 1 if delta(i, i + 1) - delta(i, i - 1) > 0 else -1
        dmin = delta(i, i - d)
        lmax = 2
        while delta(i, i + lmax * d) > dmin:
            lmax *= 2
        l, t = 0, lmax // 2
        while t >= 1:
            if delta(i, i + (l + t) * d) > dmin:
                l += t
            t //= 2
        j = i + l * d
        dn = delta(i, j)
        s, t = 0, l
        while True:
            t = (t + 1) // 2
            if delta(i, i + (s + t) * d) > dn:
                s += t
            if t == 1:
                break
        g = i + s * d + min(d, 0)
        left[i] = ~g if min(i, j) == g else g
        right[i] = ~(g + 1) if max(i, j) == g + 1 else g + 1
    return left, right


@pytest.mark.parametrize("seed,nb,ns", [(3, 2, 50), (4, 3, 300)])
def test_lbvh_matches_karras_and_prefix_property(seed, nb, ns):
    s = sg.config_blobs(seed=seed, n_blobs=nb, n_spheres=ns, subdiv=2, box=5.0)
    b = oracle.OracleScene(s).lbvh()
    keys = b["keys"]
    assert np.all(np.diff(keys.astype(np.float64)) >= 0) and len(set(keys.tolist())) == len(keys)
    kl, kr = _karras_per_node(keys)
    assert b["left"].tolist() == kl and b["right"].tolist() == kr
    # every internal node covers a range split at its highest differing bit
    n = len(keys)

    def rng_of(c):
        if c < 0:
            return ~c, ~c
        lo_a, _ = rng_of(b["left"][c])
        _, hi_b = rng_of(b["right"][c])
        return lo_a, hi_b

    import sys
    sys.setrecursionlimit(10000)
    for i in range(n - 1):
        a, z = rng_of(i)
        assert i in (a, z)
        bit = 63 - _clz64(int(keys[a]) ^ int(keys[z]))
        la, lz = rng_of(b["left"][i])
        ra, rz = rng_of(b["right"][i])
        assert la == a and rz == z and lz + 1 == ra
        assert all((int(k) >> bit) & 1 == 0 for k in keys[la:lz + 1])
        assert all((int(k) >> bit) & 1 == 1 for k in keys[ra:rz + 1])
    # parents are the inverse of the child arrays
    par = b["parent"]
    assert par[0] == -1
    for i in range(n - 1):
        for c in (b["left"][i], b["right"][i]):
            assert par[c if c >= 0 else n - 1 + ~c] == i


def _round_float(x: Fraction, up: bool) -> np.float32:
    f = np.float32(float(x))
    if up and Fraction(float(f)) < x:
        f = np.nextafter(f, np.float32(np.inf))
    if not up and Fraction(float(f)) > x:
        f = np.nextafter(f, np.float32(-np.inf))
    return f


def test_lbvh_boxes_exact_and_conservative():
    s = sg.config_blobs(seed=5, n_blobs=2, n_spheres=40, subdiv=1, box=3.0)
    s.spheres["center"][0] = (1e6, -3e-7, 0.1)      # force inexact double sums
    s.spheres["radius"][0] = 1e-3
    b = oracle.OracleScene(s).lbvh()
    order = (b["keys"] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    ns = len(s.spheres)
    for k, pid in enumerate(order):
        lo, hi = b["leaf_box"][k, :3], b["leaf_box"][k, 3:]
        if pid < ns:
            c, r = s.spheres["center"][pid], s.spheres["radius"][pid]
            for a in range(3):
                assert lo[a] == _round_float(Fraction(float(c[a])) - Fraction(float(r)), False)
                assert hi[a] == _round_float(Fraction(float(c[a])) + Fraction(float(r)), True)
        else:
            t = s.triangles[pid - ns]
            v = np.stack([t["v0"], t["v1"], t["v2"]])
            assert np.array_equal(lo, v.min(0)) and np.array_equal(hi, v.max(0))
    n = len(order)
    for i in range(n - 1):
        boxes = []
        for c in (b["left"][i], b["right"][i]):
            boxes.append(b["leaf_box"][~c] if c < 0 else b["inner_box"][c])
        u = np.concatenate([np.minimum(boxes[0][:3], boxes[1][:3]),
                            np.maximum(boxes[0][3:], boxes[1][3:])])
        assert np.array_equal(b["inner_box"][i], u)


# ------------------------------------------------------------ T9 shadows
def _shadow_scene(light_y=10.0):
    mats = [(0.5, 0.5, 0.5, 0.0), (0.9, 0.1, 0.1, 0.0)]
    return scene(spheres=[((3, 5, 0), 1.0, 1)], tris=quad_xz(-40, 40, -40, 40, 0.0, 0), mats=mats,
                 lights=[((3, light_y, 0), 1.0)], eye=(20, 20, 0), forward=(-1, -1, 0),
                 up=(-1, 1, 0), vfov=50.0, W=97, H=97, max_depth=0)


def test_shadow_of_sphere_closed_form():
    s = _shadow_scene()
    r = oracle.render(s)
    R_sh = 10.0 * 0.2 / math.sqrt(1 - 0.04)          # tangent cone: sin a = r/(hL-hc)
    n_sh = n_lit = 0
    for j in range(0, s.H, 2):
        for i in range(0, s.W, 2):
            if r["hit_id"][1, j, i] != 1 + 0 and r["hit_id"][1, j, i] != 2:
                continue                               # only ground hits (ids 1, 2)
            o, d = oracle.primary_ray(s, +1, i, j)
            p = o + d * (-o[1] / d[1])
            rho = math.hypot(p[0] - 3, p[2])
            col = r["rgb"][1, j, i]
            if rho < R_sh - 0.02:
                assert np.allclose(col, 0.5 * KA, atol=1e-12)
                n_sh += 1
            elif rho > R_sh + 0.02:
                ndl = 10.0 / math.sqrt(10.0 ** 2 + rho ** 2)
                assert np.allclose(col, 0.5 * (KA + ndl), atol=2e-4)
                n_lit += 1
    assert n_sh > 20 and n_lit > 200


def test_light_behind_surface_casts_no_shadow_rays():
    s = scene(tris=quad_xz(-40, 40, -40, 40, 0.0, 0), lights=[((0, -5, 0), 1.0)],
              eye=(0, 5, 0), forward=(0, -1, 0), up=(0, 0, -1), W=9, H=9, max_depth=2)
    r = oracle.render(s)
    assert r["rays"].tolist() == [2 * 81, 0, 0]
    assert np.allclose(r["rgb"], 0.5 * KA, atol=1e-15)


# --------------------------------------------------------- T10 reflections
@pytest.mark.parametrize("depth", [0, 1, 2, 3, 5])
def test_reflection_depth_geometric_series(depth):
    a = np.array([0.2, 0.4, 0.8])
    refl = 0.5
    tris = quad(-10, 10, -10, 10, -5.0, 0) + quad(-10, 10, -10, 10, 5.0, 0)
    s = scene(tris=tris, mats=[(*a, refl)], lights=[((0, 0, 0), 0.0)], W=1, H=1,
              max_depth=depth)
    r = oracle.render(s)
    expect = KA * a * (1 - refl ** (depth + 1))
    assert np.allclose(r["rgb"][0, 0, 0], expect, atol=1e-14)
    assert r["rays"].tolist() == [2, 2 * (depth + 1), 2 * depth]


def test_perfect_mirror_shows_background_only_after_one_bounce():
    s = scene(tris=quad(-10, 10, -10, 10, -5.0, 0), mats=[(0.3, 0.6, 0.9, 1.0)], W=1, H=1,
              max_depth=0)
    assert np.allclose(oracle.render(s)["rgb"][0, 0, 0], 0.0)
    s = s.with_view(max_depth=1)
    assert np.allclose(oracle.render(s)["rgb"][0, 0, 0], BG, atol=1e-15)


# ---------------------------------------------------- pixel list and counts
def test_pixel_list_matches_full_render():
    s = sg.config_small(2, W=64, H=48)
    osc = oracle.OracleScene(s)
    full = osc.render()
    pix = np.array([0, 5, 64 * 48 - 1, 64 * 48, 2 * 64 * 48 - 1, 1234])
    part = osc.render(pixels=pix)
    assert np.array_equal(part["rgb"], full["rgb"].reshape(-1, 3)[pix])
    assert np.array_equal(part["hit_id"], full["hit_id"].reshape(-1)[pix])
    assert part["rays"][0] == len(pix) and full["rays"][0] == 2 * 64 * 48


# ------------------------------------------- near-tie criteria (iv), (v)
# One pixel looking down -z at a large triangle in the plane z = -5 (hit
# point (0, 0, -5), normal +z, secondary origin o2 = p + 5e-4 n); the pixel
# is flagged (bit 1) when some decision of its ray tree is within relative
# 1e-5 of flipping, and not flagged 1e-3 away from the decision.
_GROUND = [((-1000.0, -1000.0, -5.0), (1000.0, -1000.0, -5.0), (0.0, 1000.0, -5.0), 0)]
_O2 = np.array([0.0, 0.0, -5.0 + 5e-4])


def _one_pixel(tris, light):
    return scene(tris=tris, mats=[(0.5, 0.5, 0.5, 0.0)], lights=[(tuple(light), 1.0)],
                 W=1, H=1, eye_sep=0.0, max_depth=0)


@pytest.mark.parametrize("c,flagged", [(1e-6, True), (-1e-6, True), (1e-3, False), (-1e-3, False)])
def test_near_tie_flag_grazing_light(c, flagged):
    """n.l = c: a light 100 away from o2 at elevation asin(c) over the plane;
    |n.l| < 1e-5 is a near tie whatever its sign (criterion (v))."""
    L = _O2 + 100.0 * np.array([math.sqrt(1.0 - c * c), 0.0, c])
    r = oracle.render(_one_pixel(_GROUND, L))
    assert r["hit_id"][0, 0, 0] == 0
    assert bool(r["flags"][0, 0, 0] & 2) == flagged, r["flags"][0, 0, 0]
    if not flagged:
        # lit when the light is above the plane, ambient only below it
        expect = 0.5 * (KA + max(c, 0.0))
        assert np.allclose(r["rgb"][0, 0, 0], expect, atol=1e-9)


@pytest.mark.parametrize("delta,flagged,lit", [(1e-6, True, None), (-1e-6, True, None),
                                               (1e-3, False, True), (-1e-3, False, False)])
def test_near_tie_flag_occluder_at_the_shadow_cutoff(delta, flagged, lit):
    """A small occluder triangle, perpendicular to the shadow ray, at distance tmax (1 + delta)
    from o2, tmax = |L - o2| - eps: within relative 1e-5 of the cut-off it is
    a near tie (criterion (iv)); 1e-3 before it blocks the light, 1e-3 past
    it does not."""
    L = np.array([3.0, 0.0, -1.0])
    lv = L - _O2
    ld = float(np.linalg.norm(lv))
    lh = lv / ld
    tmax = ld - 5e-4
    c = _O2 + lh * tmax * (1.0 + delta)
    u = np.cross(lh, [0.0, 1.0, 0.0])
    u /= np.linalg.norm(u)
    v = np.cross(lh, u)
    h = 0.005
    occ = [(tuple(c - h * u - h * v), tuple(c + h * u - h * v), tuple(c + h * v), 0)]
    r = oracle.render(_one_pixel(_GROUND + occ, L))
    assert r["hit_id"][0, 0, 0] == 0
    assert bool(r["flags"][0, 0, 0] & 2) == flagged, r["flags"][0, 0, 0]
    if lit is not None:
        ndl = float(lh[2])
        expect = 0.5 * (KA + (ndl if lit else 0.0))
        assert np.allclose(r["rgb"][0, 0, 0], expect, atol=1e-6), (r["rgb"][0, 0, 0], expect)
