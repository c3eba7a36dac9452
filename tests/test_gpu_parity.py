"""GPU path vs the FP64 oracle, element by element, through the C-ABI.

Pass criteria (tolerances of the FP32 GPU path against the FP64 oracle):
  * primary hit id equal on every pixel whose primary ray the oracle does
    not flag as a near tie (flags bit 0);
  * per-channel |RGB error| <= 2e-3 on at least 99.9 % of all pixels;
  * max |RGB error| <= 2e-2 over pixels with no flagged ray (flags == 0);
  * ray counts by kind equal up to the rays of flagged pixels;
  * LBVH keys, topology and FP32 boxes bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_1702_01530_gb300 import capi, scenegen as sg
from tests.scenes_util import quad, scene

pytestmark = pytest.mark.gpu

TOL, FRAC, MAXERR = 2e-3, 0.999, 2e-2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1702_01530_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.init()


def gpu_render(s, tree=None, **kw):
    g = capi.GpuScene(s)
    try:
        if tree is not None:
            capi.rt_scene_set_traversal(g.handle, tree)
        r = g.render(aux=True, **kw)
        capi.rt_sync_status(g.handle)
        out = {"rgb": r["rgb"].cpu().numpy(),
               "hit_id": r["hit_id"].cpu().numpy().view(np.uint32),
               "depth": r["depth"].cpu().numpy(),
               "rays": r["rays"].cpu().numpy()}
        if r.get("work") is not None:
            out["work"] = r["work"].cpu().numpy().reshape(3, 3)
        return out
    finally:
        g.close()


def check_parity(gpu, ref, n_lights, max_depth, check_rays=True, min_unflagged=0.9):
    err = np.abs(gpu["rgb"] - ref["rgb"])
    flags = ref["flags"]
    within = (err <= TOL).all(axis=-1).mean()
    assert within >= FRAC, f"only {within:.5f} of pixels within {TOL}"
    unfl = flags == 0
    assert unfl.mean() > min_unflagged
    assert err[unfl].max() <= MAXERR, f"max err on unflagged pixels {err[unfl].max()}"
    prim = (flags & 1) == 0
    bad = gpu["hit_id"][prim] != ref["hit_id"][prim]
    assert not bad.any(), f"{bad.sum()} unflagged primary hit ids differ"
    if check_rays:
        budget = int((flags != 0).sum()) * (n_lights * (max_depth + 1) + max_depth)
        assert gpu["rays"][0] == ref["rays"][0]
        assert abs(int(gpu["rays"][1]) - int(ref["rays"][1])) <= budget
        assert abs(int(gpu["rays"][2]) - int(ref["rays"][2])) <= budget
    return err


# ---------------------------------------------------------------- LBVH
def _lbvh_scenes():
    one = scene(spheres=[((0.1, 0.2, -3.0), 0.7, 0)])
    two = scene(spheres=[((0, 0, -3), 1.0, 0)], tris=[((0, 0, -5), (1, 0, -5), (0, 1, -5), 0)])
    same = scene(spheres=[((5.0, 5.0, 5.0), 0.1 + 0.01 * k, 0) for k in range(8)])
    return {
        "one": one, "two": two, "coincident": same,
        "small": sg.config_small(1),
        "polyhedra": sg.config_polyhedra(5, ground=True),
        "blobs": sg.config_blobs(3, n_blobs=20, n_spheres=100),
        "blobs_full": sg.config_blobs(2),
    }


@pytest.mark.parametrize("name", list(_lbvh_scenes()))
def test_lbvh_bit_exact(name):
    s = _lbvh_scenes()[name]
    g = capi.GpuScene(s)
    try:
        got = capi.rt_scene_get_bvh(g.handle)
    finally:
        g.close()
    ref = oracle.OracleScene(s).lbvh()
    for k in ("keys", "left", "right", "parent", "leaf_box", "inner_box"):
        assert np.array_equal(got[k], ref[k]), k


# -------------------------------------------------------------- render
@pytest.mark.parametrize("seed,W,H,D", [(1, 320, 240, 3), (2, 37, 23, 5), (3, 64, 48, 0),
                                        (4, 1, 1, 3), (5, 129, 67, 16)])
def test_small_scene_parity(seed, W, H, D):
    s = sg.config_small(seed, W=W, H=H, max_depth=D)
    gpu = gpu_render(s)
    ref = oracle.render(s)
    check_parity(gpu, ref, 1, D)


def test_zero_separation_is_bitwise_identical():
    s = sg.config_small(1).with_view(eye_sep=0.0)
    gpu = gpu_render(s)
    assert np.array_equal(gpu["rgb"][0], gpu["rgb"][1])
    assert np.array_equal(gpu["hit_id"][0], gpu["hit_id"][1])


def test_polyhedra_scene_parity():
    s = sg.config_polyhedra(5, n_lights=3, ground=True, W=200, H=150)
    check_parity(gpu_render(s), oracle.render(s), 3, s.max_depth)


@pytest.mark.parametrize("nb,ns,W,H", [(20, 100, 160, 90), (60, 300, 96, 64)])
def test_blob_scene_parity(nb, ns, W, H):
    # the box shrinks with the blob count so the density matches the full scene
    s = sg.config_blobs(2, n_blobs=nb, n_spheres=ns, W=W, H=H, box=50.0 * (nb / 200) ** (1 / 3))
    ref = oracle.render(s)
    assert (ref["hit_id"] != capi.RT_MISS_ID).mean() > 0.05
    check_parity(gpu_render(s), ref, 4, 5)


def test_mirror_pair_deep_recursion():
    a = (0.2, 0.4, 0.8)
    tris = quad(-10, 10, -10, 10, -5.0, 0) + quad(-10, 10, -10, 10, 5.0, 0)
    s = scene(tris=tris, mats=[(*a, 0.5)], lights=[((0, 0, 0), 0.3)], W=9, H=9, max_depth=16)
    gpu = gpu_render(s)
    ref = oracle.render(s)
    # the quads' shared diagonals run through the 9 diagonal pixels of each
    # eye: those exact edge hits are near ties by construction
    check_parity(gpu, ref, 1, 16, min_unflagged=0.85)
    # off-centre rays drift off the mirrors; the centre pixel bounces 16 times
    assert np.array_equal(gpu["rays"], ref["rays"]) and int(gpu["rays"][2]) >= 2 * 16


def test_single_primitive_scene():
    s = scene(spheres=[((0, 0, -5), 1.0, 0)], W=31, H=17)
    check_parity(gpu_render(s), oracle.render(s), 1, 3)


def test_work_counts_match_oracle_bvh_traversal():
    # the oracle walks its own LBVH (bit-identical to the GPU's) in the same
    # near-child-first order
    s = sg.config_blobs(5, n_blobs=10, n_spheres=50, W=96, H=64)
    gpu = gpu_render(s, count_work=True, tree=capi.RT_TREE_LBVH)
    ref = oracle.OracleScene(s).render(mode=oracle.OracleScene.MODE_BVH)
    g, r = gpu["work"].astype(np.float64), ref["work"].astype(np.float64)
    assert r[0, 0] > 1000
    rel = np.abs(g - r) / np.maximum(r, 1.0)
    assert rel.max() < 0.02, (g, r)


def test_sah_tree_is_another_tree_with_the_same_results():
    # the render tree (SAH splits over the LBVH's leaves) is a different
    # binary tree -- its walks visit other nodes -- with the same hits, depths,
    # images and ray counts (every other parity test runs on it as well)
    s = sg.config_blobs(3, n_blobs=30, n_spheres=150, W=160, H=120)
    lbvh = gpu_render(s, count_work=True, tree=capi.RT_TREE_LBVH)
    sah = gpu_render(s, count_work=True, tree=capi.RT_TREE_SAH)
    for k in ("rgb", "hit_id", "depth", "rays"):
        assert np.array_equal(lbvh[k], sah[k]), k
    assert not np.array_equal(sah["work"][:, 0], lbvh["work"][:, 0])
    # primitive tests: the same leaves behind conservative boxes
    assert 0.5 < sah["work"][:, 1:].sum() / lbvh["work"][:, 1:].sum() < 2.0


def test_sliced_sah_build_gives_the_one_block_tree():
    # the top levels of a 257k-primitive scene are built with each node sliced
    # over many blocks; with slicing off every level runs one block per node:
    # the same tree word for word
    s = sg.config_blobs(2, W=64, H=36)
    trees = []
    try:
        for slicing in (True, False):
            capi.rt_debug_set_sah_slicing(slicing)
            g = capi.GpuScene(s)
            try:
                trees.append(capi.rt_debug_get_sah_tree(g.handle))
            finally:
                g.close()
    finally:
        capi.rt_debug_set_sah_slicing(True)
    assert trees[0].shape == (s.n_prims - 1, 16)
    assert np.array_equal(trees[0], trees[1])
    # a valid binary tree over every leaf: each leaf and inner node (but the root) once
    kids = trees[0][:, 12:14].view(np.int32).ravel()
    n = trees[0].shape[0] + 1
    assert np.array_equal(np.sort(~kids[kids < 0]), np.arange(n))
    assert np.array_equal(np.sort(kids[kids >= 0]), np.arange(1, n - 1))


def test_host_render_matches_device_render():
    import torch
    s = sg.config_small(2, W=80, H=60)
    g = capi.GpuScene(s)
    try:
        dev = g.render()["rgb"].cpu().numpy()
        hl = torch.empty((60, 80, 3), dtype=torch.float32).pin_memory()
        hr = torch.empty((60, 80, 3), dtype=torch.float32).pin_memory()
        capi.rt_render_stereo_host(g.handle, s.camera, s.eye_sep, s.convergence, 80, 60,
                                   s.max_depth, hl, hr)
        assert np.array_equal(dev[0], hl.numpy()) and np.array_equal(dev[1], hr.numpy())
        # pageable numpy buffers take the copy path
        pl = np.zeros((60, 80, 3), np.float32)
        pr = np.zeros((60, 80, 3), np.float32)
        capi.rt_render_stereo_host(g.handle, s.camera, s.eye_sep, s.convergence, 80, 60,
                                   s.max_depth, pl, pr)
        assert np.array_equal(dev[0], pl) and np.array_equal(dev[1], pr)
    finally:
        g.close()


@pytest.mark.parametrize("make", [lambda: sg.config_blobs(3, n_blobs=30, n_spheres=150, W=128, H=96),
                                  lambda: sg.config_small(4, W=97, H=61),
                                  lambda: scene(spheres=[((0, 0, -5), 1.0, 0)], W=16, H=9),
                                  lambda: sg.config_polyhedra(6, n_lights=2, ground=True, W=80, H=60)])
def test_all_trees_give_identical_images(make):
    s = make()
    g = capi.GpuScene(s)
    try:
        sah = g.render(aux=True)                          # the default tree
        out = {}
        for tree in (capi.RT_TREE_WIDE, capi.RT_TREE_LBVH, capi.RT_TREE_SAH):
            capi.rt_scene_set_traversal(g.handle, tree)
            out[tree] = g.render(aux=True)
        capi.rt_sync_status(g.handle)
        for tree, r in out.items():
            for k in ("rgb", "hit_id", "depth", "rays"):
                assert np.array_equal(r[k].cpu().numpy(), sah[k].cpu().numpy()), (tree, k)
        with pytest.raises(capi.RtError):
            capi.rt_scene_set_traversal(g.handle, 3)
    finally:
        g.close()


def test_repeated_renders_are_identical():
    s = sg.config_blobs(4, n_blobs=10, n_spheres=40, W=64, H=48)
    g = capi.GpuScene(s)
    try:
        a = g.render()["rgb"].cpu().numpy()
        g.render(W=32, H=16)
        b = g.render()["rgb"].cpu().numpy()
        assert np.array_equal(a, b)
    finally:
        g.close()


# ------------------------------------------------ sequences to the host
def test_sequence_to_host_equals_single_renders():
    # one pair per camera, copies overlapped with the next render; a host
    # buffer named for several frames ends up with the last of them
    import torch
    s = sg.config_blobs(3, n_blobs=12, n_spheres=60, W=160, H=96)
    cams = []
    for dx in (0.0, 1.5, -2.0, 0.5, 3.0):
        c = s.camera.copy()
        c["eye"][0] += dx
        cams.append(c)
    g = capi.GpuScene(s)
    try:
        ref = []
        for c in cams:
            out = torch.empty((2, s.H, s.W, 3), dtype=torch.float32, device="cuda")
            capi.rt_render_stereo(g.handle, c, s.eye_sep, s.convergence, s.W, s.H, s.max_depth,
                                  out[0], out[1])
            ref.append(out.cpu().numpy())
        capi.rt_sync_status(g.handle)
        own = [torch.empty((2, s.H, s.W, 3), dtype=torch.float32).pin_memory() for _ in cams]
        capi.rt_render_stereo_sequence(g.handle, cams, s.eye_sep, s.convergence, s.W, s.H,
                                       s.max_depth, [o[0] for o in own], [o[1] for o in own])
        for f in range(len(cams)):
            assert np.array_equal(own[f].numpy(), ref[f]), f
        ring = [torch.empty((2, s.H, s.W, 3), dtype=torch.float32).pin_memory() for _ in range(2)]
        capi.rt_render_stereo_sequence(g.handle, cams, s.eye_sep, s.convergence, s.W, s.H,
                                       s.max_depth, [ring[f % 2][0] for f in range(len(cams))],
                                       [ring[f % 2][1] for f in range(len(cams))])
        assert np.array_equal(ring[0].numpy(), ref[4]) and np.array_equal(ring[1].numpy(), ref[3])
        unpinned = [np.zeros((2, s.H, s.W, 3), np.float32) for _ in range(2)]
        capi.rt_render_stereo_sequence(g.handle, cams[:2], s.eye_sep, s.convergence, s.W, s.H,
                                       s.max_depth, [u[0] for u in unpinned],
                                       [u[1] for u in unpinned])
        assert np.array_equal(unpinned[1], ref[1])
        bad = cams[:2]
        bad[1] = bad[1].copy()
        bad[1]["vfov_deg"] = 0.0
        with pytest.raises(capi.RtError) as e:
            capi.rt_render_stereo_sequence(g.handle, bad, s.eye_sep, s.convergence, s.W, s.H,
                                           s.max_depth, [u[0] for u in unpinned],
                                           [u[1] for u in unpinned])
        assert e.value.code == capi.RT_ERR_INVALID_ARG
        capi.rt_sync_status(g.handle)
    finally:
        g.close()


# ------------------------------------------------------- drain pools
def test_blob_pair_renders_are_identical_at_full_size():
    # the end of every frame hands queued rays between warps through the
    # drain pools: a ray lost or traced twice would change the fixed-point sums
    s = sg.config_blobs(2)
    g = capi.GpuScene(s)
    try:
        first = g.render(aux=True)
        ref_rgb, ref_rays = first["rgb"].cpu().numpy(), first["rays"].cpu().numpy()
        for _ in range(4):
            r = g.render(aux=True)
            assert np.array_equal(r["rgb"].cpu().numpy(), ref_rgb)
            assert np.array_equal(r["rays"].cpu().numpy(), ref_rays)
        capi.rt_sync_status(g.handle)
    finally:
        g.close()


@pytest.mark.parametrize("cap", [1, 37, 4096])
def test_full_drain_pools_fall_back_to_the_owning_warp(cap):
    # pools too small for the frame: the rays that do not fit stay with the
    # warp that queued them (and the pool ends with empty entries); the image
    # and the ray counts must not change
    s = sg.config_blobs(3, n_blobs=30, n_spheres=150, W=256, H=192)
    g = capi.GpuScene(s)
    try:
        ref = g.render(aux=True)
        capi.rt_debug_set_pool_capacity(g.handle, cap)
        small = g.render(aux=True)
        capi.rt_sync_status(g.handle)
        for k in ("rgb", "hit_id", "rays"):
            assert np.array_equal(small[k].cpu().numpy(), ref[k].cpu().numpy()), k
        capi.rt_debug_set_pool_capacity(g.handle, 0)
        again = g.render(aux=True)
        assert np.array_equal(again["rgb"].cpu().numpy(), ref["rgb"].cpu().numpy())
    finally:
        g.close()


# ---------------------------------------------- full size, sampled pixels
def test_full_size_blob_scene_sampled_parity():
    """256,000 triangles + 1,000 spheres at 1920x1080 per eye, depth 5, 4
    lights, rendered exactly as the benchmark renders it; the oracle traces
    a seeded sample of pixels one by one."""
    import torch
    s = sg.config_blobs(2)
    g = capi.GpuScene(s)
    try:
        img = g.render()["rgb"]                      # the timed call
        aux = g.render(aux=True)                     # same image + hit ids
        capi.rt_sync_status(g.handle)
        assert torch.equal(img, aux["rgb"])
        rgb = aux["rgb"].cpu().numpy().reshape(-1, 3)
        hit = aux["hit_id"].cpu().numpy().view(np.uint32).reshape(-1)
    finally:
        g.close()
    rng = np.random.default_rng(2024)
    pix = rng.choice(2 * s.W * s.H, size=3000, replace=False)
    ref = oracle.OracleScene(s).render(pixels=pix)
    err = np.abs(rgb[pix] - ref["rgb"])
    assert (err <= TOL).all(axis=-1).mean() >= FRAC
    unfl = ref["flags"] == 0
    assert err[unfl].max() <= MAXERR
    prim = (ref["flags"] & 1) == 0
    assert np.array_equal(hit[pix][prim], ref["hit_id"][prim])
    assert (ref["hit_id"] != capi.RT_MISS_ID).mean() > 0.05


def test_terrain_parity_small_grid():
    # the terrain recipe on a 65 x 65 grid (8,192 triangles) with 40 spheres
    s = sg.config_terrain(n_grid=65, n_spheres=40, W=96, H=54)
    ref = oracle.render(s)
    assert (ref["hit_id"] != capi.RT_MISS_ID).mean() > 0.5
    check_parity(gpu_render(s), ref, 8, s.max_depth)


def test_full_size_terrain_sampled_parity():
    """9,990,450 triangles + 10,000 spheres at 3840x2160 per eye, depth 4, 8
    lights: frame 0 of the terrain sequence, rendered as the sequence renders
    it; the oracle traces a seeded sample of pixels one by one."""
    s = sg.config_terrain()
    g = capi.GpuScene(s)
    try:
        aux = g.render(aux=True)
        capi.rt_sync_status(g.handle)
        rgb = aux["rgb"].cpu().numpy().reshape(-1, 3)
        hit = aux["hit_id"].cpu().numpy().view(np.uint32).reshape(-1)
    finally:
        g.close()
    rng = np.random.default_rng(2025)
    pix = rng.choice(2 * s.W * s.H, size=2000, replace=False)
    ref = oracle.OracleScene(s).render(pixels=pix)
    err = np.abs(rgb[pix] - ref["rgb"])
    assert (err <= TOL).all(axis=-1).mean() >= FRAC
    unfl = ref["flags"] == 0
    assert unfl.mean() > 0.9 and err[unfl].max() <= MAXERR
    prim = (ref["flags"] & 1) == 0
    assert np.array_equal(hit[pix][prim], ref["hit_id"][prim])
    assert (ref["hit_id"] != capi.RT_MISS_ID).mean() > 0.5


# ------------------------------------------------------------ watchdog
def test_bvh_cycle_stops_at_iteration_bound():
    s = sg.config_blobs(6, n_blobs=2, n_spheres=20, W=32, H=24, max_depth=1)
    g = capi.GpuScene(s)
    try:
        bvh = capi.rt_scene_get_bvh(g.handle)
        # node 0 becomes its own left child; its right child gets an empty
        # box: every ray entering the root loops until the iteration bound
        capi.rt_debug_set_node(g.handle, 0, 0, int(bvh["right"][0]), empty_right=True)
        capi.rt_scene_set_traversal(g.handle, capi.RT_TREE_LBVH)   # the hook edits the LBVH
        g.render()
        with pytest.raises(capi.RtError) as e:
            capi.rt_sync_status(g.handle)
        assert e.value.code == capi.RT_ERR_TIMEOUT
        capi.rt_sync_status(g.handle)                # cleared after reporting
    finally:
        g.close()
    gpu = gpu_render(sg.config_small(1, W=32, H=24))  # the context is still usable
    assert gpu["rgb"].shape == (2, 24, 32, 3)


@pytest.mark.parametrize("n_prims", [1023, 1024])
def test_pair_eyes_cutoff_both_sides(n_prims):
    """Scenes of 1024 or more primitives trace a pixel's two eyes in
    neighbouring lanes (4x4-pixel tiles), smaller ones 8x4 tiles of one eye:
    parity on both sides of the cut-off at an odd size, and a zero
    separation gives identical eyes bit for bit on both sides."""
    rng = np.random.default_rng(77)
    sph = []
    for k in range(n_prims):
        c = (float(rng.uniform(-30, 30)), float(rng.uniform(-7, 7)), float(rng.uniform(-20, -8)))
        sph.append((c, float(rng.uniform(0.3, 1.0)), k % 3))
    mats = [(0.8, 0.3, 0.2, 0.0), (0.2, 0.7, 0.3, 0.0), (0.6, 0.6, 0.6, 0.5)]
    s = scene(spheres=sph, mats=mats, lights=[((3.0, 10.0, 0.0), 1.0)], W=33, H=9,
              eye_sep=0.065, convergence=15.0, max_depth=3)
    assert s.n_prims == n_prims
    ref = oracle.render(s)
    assert (ref["hit_id"] != capi.RT_MISS_ID).mean() > 0.5
    check_parity(gpu_render(s), ref, 1, 3)
    z = gpu_render(s.with_view(eye_sep=0.0))
    assert np.array_equal(z["rgb"][0], z["rgb"][1])
    assert np.array_equal(z["hit_id"][0], z["hit_id"][1])
