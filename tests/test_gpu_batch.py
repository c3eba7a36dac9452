"""Batched stereo rendering on the GPU, through the C-ABI.

* every request of a batch (uneven resolutions incl. 1x1 and ragged tiles,
  also for a scene whose single renders trace both eyes of a pixel in one warp,
  depths 0-6, several scenes, one scene under two cameras) equals the
  single-pair rt_render_stereo of the same arguments bit for bit, for every
  tile shape, request order, mirror-queue capacity and residency;
* one request of a batch against the FP64 oracle with the parity criteria;
* ray counts equal the single renders' sums; per-request latencies are
  positive and inside the launch;
* a camera changed between launches takes effect; the autotuner keeps a
  valid configuration and the images do not change.
"""
import numpy as np
import pytest

import oracle
from paper_1702_01530_gb300 import capi, scenegen as sg
from tests.test_gpu_parity import check_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1702_01530_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.init()


def _scenes():
    return [sg.config_small(1),
            sg.config_polyhedra(5, n_lights=3, ground=True),
            sg.config_blobs(5, n_blobs=12, n_spheres=60, max_depth=6,
                            box=50.0 * (12 / 200) ** (1 / 3))]


# (scene index, W, H, max_depth, eye_sep, camera shift along x)
_REQS = [(0, 320, 240, 3, 0.065, 0.0), (1, 203, 77, 2, 0.2, 0.0), (2, 160, 90, 6, 0.065, 0.0),
         (0, 1, 1, 3, 0.065, 0.0), (2, 33, 9, 0, 0.5, 0.0), (0, 97, 61, 5, 0.065, 1.5),
         (1, 64, 64, 4, 0.0, 0.0), (2, 1, 1, 4, 0.065, 0.0), (2, 3, 2, 5, 0.3, 0.0)]


class _Fixture:
    def __init__(self, reqs=_REQS):
        import torch
        self.scenes = _scenes()
        self.g = [capi.GpuScene(s) for s in self.scenes]
        self.items, self.outs, self.args = [], [], []
        for si, W, H, D, es, dx in reqs:
            s = self.scenes[si]
            cam = s.camera.copy()
            cam["eye"][0] += dx
            o = torch.full((2, H, W, 3), -1.0, dtype=torch.float32, device="cuda")
            self.outs.append(o)
            self.args.append((si, cam, es, s.convergence, W, H, D))
            self.items.append((self.g[si].handle, cam, es, s.convergence, W, H, D, o[0], o[1]))
        self.reqs = capi.make_requests(self.items)

    def single(self, i, cam=None):
        """rt_render_stereo_aux of request i (optionally under another camera)."""
        import torch
        si, cam0, es, cv, W, H, D = self.args[i]
        cam = cam0 if cam is None else cam
        img = torch.empty((2, H, W, 3), dtype=torch.float32, device="cuda")
        rays = torch.zeros(3, dtype=torch.int64, device="cuda")
        hit = torch.empty((2, H, W), dtype=torch.int32, device="cuda")
        dep = torch.empty((2, H, W), dtype=torch.float32, device="cuda")
        capi.rt_render_stereo_aux(self.g[si].handle, cam, es, cv, W, H, D, img[0], img[1], hit[0],
                                  hit[1], dep[0], dep[1], rays, None)
        capi.rt_sync_status(self.g[si].handle)
        return {"img": img, "hit_id": hit.cpu().numpy().view(np.uint32),
                "rays": rays.cpu().numpy()}

    def close(self):
        for g in self.g:
            g.close()


@pytest.fixture(scope="module")
def fx():
    f = _Fixture()
    f.ref = [(r["img"], r["rays"]) for r in (f.single(i) for i in range(len(_REQS)))]
    yield f
    f.close()


def _run(fx, cfg=None):
    import torch
    for o in fx.outs:
        o.fill_(-1.0)
    b = capi.rt_batch_create(fx.reqs, cfg)
    try:
        capi.rt_batch_launch(b)
        rays, lat, c = capi.rt_batch_stats(b, len(fx.outs))
    finally:
        capi.rt_batch_destroy(b)
    torch.cuda.synchronize()
    return rays, lat, c


def test_batch_equals_single_renders_bitwise(fx):
    import torch
    rays, lat, c = _run(fx)
    for i, (img, _) in enumerate(fx.ref):
        assert torch.equal(fx.outs[i], img), f"request {i} differs"
    want = np.sum([r for _, r in fx.ref], axis=0)
    assert rays.tolist() == want.tolist()
    assert (lat > 0).all()
    assert (c["tile_w"][0], c["tile_h"][0]) == (4, 4) and c["blocks_per_sm"][0] >= 1


@pytest.mark.parametrize("tile", [(8, 2), (2, 8), (16, 1), (8, 4), (4, 8), (32, 1)])
@pytest.mark.parametrize("order", [capi.RT_BATCH_ORDER_GIVEN, capi.RT_BATCH_ORDER_SMALLEST_FIRST])
def test_batch_configurations_give_identical_images(fx, tile, order):
    import torch
    cfg = capi.batch_config(tile_w=tile[0], tile_h=tile[1], order=order, cap_r=128,
                            blocks_per_sm=3, track_latency=0)
    rays, lat, c = _run(fx, cfg)
    for i, (img, _) in enumerate(fx.ref):
        assert torch.equal(fx.outs[i], img), f"request {i} differs"
    assert (lat == -1).all()
    assert int(c["blocks_per_sm"][0]) == 3 and int(c["cap_r"][0]) == 128


def test_batch_request_against_oracle(fx):
    # request 0: the small scene at 320x240, depth 3, straight from the batch
    _run(fx)
    s = fx.scenes[0]
    ref = oracle.render(s)
    single = fx.single(0)
    gpu = {"rgb": fx.outs[0].cpu().numpy(), "hit_id": single["hit_id"], "rays": single["rays"]}
    check_parity(gpu, ref, 1, s.max_depth)


def test_batch_set_camera_and_relaunch(fx):
    import torch
    b = capi.rt_batch_create(fx.reqs)
    try:
        capi.rt_batch_launch(b)
        cam = fx.args[2][1].copy()
        cam["eye"][1] += 2.0
        cam["forward"][0] = 0.2
        capi.rt_batch_set_camera(b, 2, cam, 0.1, 70.0)
        capi.rt_batch_launch(b)
        capi.rt_batch_stats(b, len(fx.outs))
        torch.cuda.synchronize()
        si, _, _, _, W, H, D = fx.args[2]
        img = torch.empty((2, H, W, 3), dtype=torch.float32, device="cuda")
        capi.rt_render_stereo(fx.g[si].handle, cam, 0.1, 70.0, W, H, D, img[0], img[1])
        capi.rt_sync_status(fx.g[si].handle)
        assert torch.equal(fx.outs[2], img)
        assert not torch.equal(fx.outs[2], fx.ref[2][0])
        for i in (0, 1, 3):
            assert torch.equal(fx.outs[i], fx.ref[i][0])
    finally:
        capi.rt_batch_destroy(b)


def test_batch_autotune_keeps_images(fx):
    import torch
    b = capi.rt_batch_create(fx.reqs)
    try:
        cfg, ms = capi.rt_batch_autotune(b, reps=2)
        assert ms > 0
        assert int(cfg["tile_w"][0]) * int(cfg["tile_h"][0]) in (16, 32)
        assert int(cfg["cap_r"][0]) in (64, 128, 256)
        capi.rt_batch_launch(b)
        rays, lat, c = capi.rt_batch_stats(b, len(fx.outs))
        assert np.array_equal(c, cfg)
    finally:
        capi.rt_batch_destroy(b)
    torch.cuda.synchronize()
    for i, (img, _) in enumerate(fx.ref):
        assert torch.equal(fx.outs[i], img), f"request {i} differs"


def test_batch_latency_within_launch(fx):
    import torch
    b = capi.rt_batch_create(fx.reqs)
    try:
        capi.rt_batch_launch(b)
        capi.rt_batch_stats(b, len(fx.outs))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        st = torch.cuda.current_stream()
        e0.record(st)
        capi.rt_batch_launch(b, st)
        e1.record(st)
        e1.synchronize()
        total = e0.elapsed_time(e1)
        _, lat, _ = capi.rt_batch_stats(b, len(fx.outs))
    finally:
        capi.rt_batch_destroy(b)
    assert (lat > 0).all() and lat.max() <= total + 0.05, (lat, total)


def test_batch_rejects_bad_arguments(fx):
    bad = capi.batch_config(tile_w=5, tile_h=6)
    with pytest.raises(capi.RtError) as e:
        capi.rt_batch_create(fx.reqs, bad)
    assert e.value.code == capi.RT_ERR_INVALID_ARG
    big = capi.make_requests([(fx.g[0].handle, fx.scenes[0].camera, 0.065, 10.0, 32768, 32768, 1,
                               16, 16)] * 3)
    with pytest.raises(capi.RtError) as e:
        capi.rt_batch_create(big)
    assert e.value.code == capi.RT_ERR_INVALID_ARG
    r = fx.reqs.copy()
    r["max_depth"][1] = 17
    with pytest.raises(capi.RtError):
        capi.rt_batch_create(r)
