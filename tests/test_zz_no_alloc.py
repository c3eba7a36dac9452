"""rt_build_lbvh_noalloc: the BVH build for callers that may not allocate.

Some users of this library cannot call cudaMalloc -- for example a plugin
whose host application owns all GPU memory through its own pool, or a
real-time loop that must not pay for cudaMalloc's implicit device
synchronisation. rt_build_lbvh_noalloc serves them: the caller passes its
own device buffers and the scratch lives in a static device array. This
file checks, through the C-ABI, that two builds in a row (a larger scene,
then a smaller one, so stale scratch from the first call is present) give
exactly the BVH of rt_scene_create, and that oversized builds are refused.
It is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1702_01530_gb300 import capi, scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1702_01530_gb300 import build
    build.build()


def _child_box(nodes, i, slot):
    f = nodes[16 * i: 16 * i + 16]
    if slot == 0:
        return np.array([f[0], f[2], f[8], f[1], f[3], f[9]], np.float32)
    return np.array([f[4], f[6], f[10], f[5], f[7], f[11]], np.float32)


def _noalloc_build(s):
    import torch
    n = s.n_prims
    ns, nt = len(s.spheres), len(s.triangles)
    sp = torch.from_numpy(np.ascontiguousarray(s.spheres).view(np.uint8).copy()).cuda() if ns else None
    tr = torch.from_numpy(np.ascontiguousarray(s.triangles).view(np.uint8).copy()).cuda() if nt else None
    nodes = torch.full((max(n - 1, 1) * 16,), -7.0, dtype=torch.float32, device="cuda")
    prims = torch.full((n * 12,), -7.0, dtype=torch.float32, device="cuda")
    keys = torch.zeros(n, dtype=torch.int64, device="cuda")
    parent = torch.zeros(2 * n - 1, dtype=torch.int32, device="cuda")
    capi.rt_build_lbvh_noalloc(sp, ns, tr, nt, nodes, prims, keys, parent)
    nodes = nodes.cpu().numpy()
    out = {"keys": keys.cpu().numpy().view(np.uint64), "parent": parent.cpu().numpy(),
           "prims": prims.cpu().numpy().reshape(n, 12)}
    ints = nodes.view(np.int32)
    left = np.array([ints[16 * i + 12] for i in range(n - 1)], np.int32)
    right = np.array([ints[16 * i + 13] for i in range(n - 1)], np.int32)
    leaf_box = np.zeros((n, 6), np.float32)
    inner_box = np.zeros((max(n - 1, 0), 6), np.float32)
    for i in range(n - 1):
        for slot, c in ((0, left[i]), (1, right[i])):
            (leaf_box[~c] if c < 0 else inner_box[c])[:] = _child_box(nodes, i, slot)
    if n > 1:
        b0, b1 = _child_box(nodes, 0, 0), _child_box(nodes, 0, 1)
        inner_box[0] = np.concatenate([np.minimum(b0[:3], b1[:3]), np.maximum(b0[3:], b1[3:])])
    else:
        leaf_box[0] = _child_box(nodes, 0, 0)
    out.update(left=left, right=right, leaf_box=leaf_box, inner_box=inner_box)
    return out


def _expected_prims(s, keys):
    """Leaf records rebuilt on the host from the scene arrays (layout of the
    renderer: triangle v0|id, v1-v0|material, v2-v0|0; sphere c|id,
    r,0,0|material, zeros)."""
    ns = len(s.spheres)
    out = np.zeros((len(keys), 12), np.float32)
    ints = out.view(np.uint32)
    for k, key in enumerate(keys):
        pid = int(key) & 0xFFFFFFFF
        if pid < ns:
            sp = s.spheres[pid]
            out[k, 0:3] = sp["center"]
            out[k, 4] = sp["radius"]
            ints[k, 7] = sp["material"]
        else:
            t = s.triangles[pid - ns]
            out[k, 0:3] = t["v0"]
            out[k, 4:7] = t["v1"] - t["v0"]
            out[k, 8:11] = t["v2"] - t["v0"]
            ints[k, 7] = t["material"]
        ints[k, 3] = pid
    return out


def test_noalloc_build_matches_scene_create_twice_in_a_row():
    scenes = [sg.config_blobs(3, n_blobs=20, n_spheres=100), sg.config_small(1)]
    for s in scenes:                                  # two calls in a row
        got = _noalloc_build(s)
        g = capi.GpuScene(s)
        try:
            ref = capi.rt_scene_get_bvh(g.handle)
        finally:
            g.close()
        for k in ("keys", "left", "right", "parent", "leaf_box", "inner_box"):
            assert np.array_equal(got[k], ref[k]), k
        assert np.array_equal(got["prims"].view(np.uint32),
                              _expected_prims(s, got["keys"]).view(np.uint32))


def test_noalloc_build_rejects_sizes_beyond_its_limit():
    with pytest.raises(capi.RtError) as e:
        capi.rt_build_lbvh_noalloc(16, (1 << 20) + 1, None, 0, 16, 16, 16, 16)
    assert e.value.code == capi.RT_ERR_INVALID_ARG and "limit" in str(e.value)


def _bvh_arrays(nodes, n):
    """keys-free BVH arrays (left, right, leaf and inner boxes) from raw
    64-byte nodes, vectorised for large trees."""
    f = nodes.reshape(max(n - 1, 1), 16)[:n - 1]
    ints = f.view(np.int32)
    left, right = ints[:, 12].copy(), ints[:, 13].copy()
    box0 = f[:, [0, 2, 8, 1, 3, 9]]
    box1 = f[:, [4, 6, 10, 5, 7, 11]]
    leaf_box = np.zeros((n, 6), np.float32)
    inner_box = np.zeros((n - 1, 6), np.float32)
    for c, b in ((left, box0), (right, box1)):
        lf = c < 0
        leaf_box[~c[lf]] = b[lf]
        inner_box[c[~lf]] = b[~lf]
    inner_box[0] = np.concatenate([np.minimum(box0[0, :3], box1[0, :3]),
                                   np.maximum(box0[0, 3:], box1[0, 3:])])
    return dict(left=left, right=right, leaf_box=leaf_box, inner_box=inner_box)


def test_noalloc_build_near_its_limit():
    """A terrain grid of 725 x 725 heights: 1,048,352 triangles, 224 short of
    the 2^20-primitive limit, so the scratch array holds the largest build it
    admits; the tree equals rt_scene_create's bit for bit."""
    import torch
    s = sg.config_terrain(5, n_grid=725, n_spheres=0, n_lights=1, W=64, H=36)
    n = s.n_prims
    assert (1 << 20) - 256 < n <= (1 << 20)
    tr = torch.from_numpy(np.ascontiguousarray(s.triangles).view(np.uint8).copy()).cuda()
    nodes = torch.full(((n - 1) * 16,), -7.0, dtype=torch.float32, device="cuda")
    prims = torch.full((n * 12,), -7.0, dtype=torch.float32, device="cuda")
    keys = torch.zeros(n, dtype=torch.int64, device="cuda")
    parent = torch.zeros(2 * n - 1, dtype=torch.int32, device="cuda")
    capi.rt_build_lbvh_noalloc(None, 0, tr, n, nodes, prims, keys, parent)
    got = _bvh_arrays(nodes.cpu().numpy(), n)
    got.update(keys=keys.cpu().numpy().view(np.uint64), parent=parent.cpu().numpy())
    g = capi.GpuScene(s)
    try:
        ref = capi.rt_scene_get_bvh(g.handle)
    finally:
        g.close()
    for k in ("keys", "left", "right", "parent", "leaf_box", "inner_box"):
        assert np.array_equal(got[k], ref[k]), k
