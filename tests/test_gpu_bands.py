"""Row-band split of a stereo pair (paper Sec. 3, Figure 1: each processor
renders one part of the image): bands rendered by rt_render_stereo_rows and
stitched in row order equal the whole pair of rt_render_stereo bit for bit,
for bands of any height (including 1 row and heights that are no multiple
of the 4-row tiles) and both tile layouts (scenes below and above the
1024-primitive cut-off for tracing a pixel's two eyes in one warp)."""
import numpy as np
import pytest

from paper_1702_01530_gb300 import bands, capi, scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1702_01530_gb300 import build
    build.build()
    torch.cuda.init()


def _stitched(s, parts):
    import torch
    g = capi.GpuScene(s)
    try:
        full = g.render(aux=True)
        L = torch.empty((s.H, s.W, 3), dtype=torch.float32, device="cuda")
        R = torch.empty_like(L)
        rays = np.zeros(3, np.int64)
        for r0, k in parts:
            bl = torch.full((k, s.W, 3), -1.0, dtype=torch.float32, device="cuda")
            br = torch.full_like(bl, -1.0)
            rc = torch.zeros(3, dtype=torch.int64, device="cuda")
            capi.rt_render_stereo_rows(g.handle, s.camera, s.eye_sep, s.convergence, s.W, s.H,
                                       s.max_depth, r0, k, bl, br, rc)
            L[r0:r0 + k], R[r0:r0 + k] = bl, br
            rays += rc.cpu().numpy()
        capi.rt_sync_status(g.handle)
        return full, L, R, rays
    finally:
        g.close()


@pytest.mark.parametrize("n", [1, 2, 3, 7])
def test_bands_stitch_to_the_full_pair_small_scene(n):
    s = sg.config_small(3, W=97, H=61)
    full, L, R, rays = _stitched(s, bands.row_bands(s.H, n))
    assert np.array_equal(L.cpu().numpy(), full["rgb"][0].cpu().numpy())
    assert np.array_equal(R.cpu().numpy(), full["rgb"][1].cpu().numpy())
    assert np.array_equal(rays, full["rays"].cpu().numpy())


def test_bands_stitch_to_the_full_pair_blob_scene_uneven_bands():
    s = sg.config_blobs(3, n_blobs=20, n_spheres=100, W=160, H=90)
    assert s.n_prims >= 1024                     # both eyes of a pixel in one warp
    parts = [(0, 1), (1, 5), (6, 33), (39, 2), (41, 49)]
    full, L, R, rays = _stitched(s, parts)
    assert np.array_equal(L.cpu().numpy(), full["rgb"][0].cpu().numpy())
    assert np.array_equal(R.cpu().numpy(), full["rgb"][1].cpu().numpy())
    assert np.array_equal(rays, full["rays"].cpu().numpy())


def test_band_arguments_checked():
    import torch
    s = sg.config_small(1, W=16, H=8)
    g = capi.GpuScene(s)
    try:
        b = torch.empty((8, 16, 3), dtype=torch.float32, device="cuda")
        for r0, k in ((0, 0), (8, 1), (5, 4)):
            with pytest.raises(capi.RtError) as e:
                capi.rt_render_stereo_rows(g.handle, s.camera, s.eye_sep, s.convergence, 16, 8,
                                           3, r0, k, b, b)
            assert e.value.code == capi.RT_ERR_INVALID_ARG
    finally:
        g.close()
