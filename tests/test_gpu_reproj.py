"""Learned reprojection on the GPU vs the oracle, through the C-ABI.

* forward warp: hole mask and source pixels exact (the target column is an
  integer decided in float32 on both sides), features within 1e-6;
* network forward (tcgen05, BF16 operands, FP32 accumulation): within 5e-3 of
  the float64 oracle that rounds to BF16 at the same points;
* gradients (tensor-core data gradients with BF16 intermediates, FP32 weight
  gradients): relative L2 error per tensor <= 1e-2 against a float64
  backward pass that rounds to BF16 at the same points, and cosine > 0.99
  against plain float64 autograd;
* the reprojected pair equals the full trace bit for bit when every right
  pixel is retraced, and its left image always equals the full trace's.
"""
import numpy as np
import pytest

from oracle import reproj as orp
from paper_1702_01530_gb300 import capi, scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1702_01530_gb300 import build
    build.build()
    torch.cuda.init()


def _t(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


@pytest.mark.parametrize("W,H,seed", [(97, 41, 1), (256, 3, 2), (1, 5, 3), (333, 20, 4)])
def test_warp_matches_oracle(W, H, seed):
    import torch
    depth, normal, ids, rgb, refl = sg.gbuffer_synthetic(seed, W, H)
    f_px, s, zc = 731.25, 0.065 * 3, 9.0
    P = W * H
    zbuf = torch.empty(P, dtype=torch.int64, device="cuda")
    f16 = torch.empty((P, 16), dtype=torch.bfloat16, device="cuda")
    f32 = torch.empty((P, orp.IN_CH), dtype=torch.float32, device="cuda")
    hole = torch.empty(P, dtype=torch.uint8, device="cuda")
    warped = torch.empty((P, 3), dtype=torch.float32, device="cuda")
    capi.rt_reproj_warp(_t(depth), _t(normal), _t(ids.view(np.int32)), _t(rgb), W, H, f_px, s, zc,
                        zbuf, f16, f32, hole, warped, refl_L=_t(refl))
    torch.cuda.synchronize()
    feat, ohole, owarp, src = orp.warp(depth, normal, ids, rgb, W, H, f_px, s, zc, refl)
    hc = hole.cpu().numpy()
    assert np.array_equal(hc == 1, ohole)
    # 2 marks a right pixel whose source surface reflects (always retraced)
    assert np.array_equal(hc == 2, ~ohole & (feat[:, 9] > 0))
    g = f32.cpu().numpy()
    assert np.abs(g - feat).max() <= 1e-6
    assert np.abs(warped.cpu().numpy() - owarp).max() <= 1e-7
    c = orp.IN_CH
    assert torch.equal(f16[:, :c].float(), f32.to(torch.bfloat16).float()) and (f16[:, c:] == 0).all()
    assert (feat[~ohole, 9] > 0).any() or (~ohole).sum() < 10  # the reflectivity channel is carried
    assert 0 < ohole.mean() < 1 or P < 10


@pytest.mark.parametrize("W,H", [(300, 7), (128, 2), (1, 3), (1000, 5)])
def test_network_forward_matches_oracle(W, H):
    import torch
    params = sg.net_params_he(11)
    rng = np.random.default_rng(5)
    params[orp.OFF_B[0]:orp.OFF_B[0] + 32] = rng.normal(0, 0.1, 32)             # non-zero biases
    params[orp.OFF_B[3]] = -0.5
    feat = sg.bf16_features_synthetic(12, W, H)
    net = capi.Net(params)
    try:
        prob = torch.empty(W * H, dtype=torch.float32, device="cuda")
        capi.rt_net_forward(net.handle, _t(feat, torch.bfloat16), W, H, prob)
        capi.rt_net_status(net.handle)
        got = prob.cpu().numpy().reshape(H, W)
    finally:
        net.close()
    ref = orp.forward(params, feat, W, H, bf16=True)
    err = np.abs(got - ref)
    assert err.max() <= 5e-3 and err.mean() <= 2e-4, (err.max(), err.mean())
    assert ref.std() > 1e-3


def test_gradients_match_float64_autograd():
    import torch
    W, H = 200, 9
    params = sg.net_params_he(21)
    params[orp.OFF_B[3]] = 0.2
    feat = sg.bf16_features_synthetic(22, W, H)
    label = (np.random.default_rng(6).random(W * H) < 0.3).astype(np.float32)
    net = capi.Net(params)
    try:
        grads = torch.zeros(capi.RT_NET_PARAMS, dtype=torch.float32, device="cuda")
        loss = capi.rt_net_train_step(net.handle, _t(feat, torch.bfloat16), _t(label), W, H, 0.0,
                                      grads=grads)
        capi.rt_net_status(net.handle)
        g = grads.cpu().numpy().astype(np.float64)
        assert np.array_equal(net.params(), params)        # lr = 0: no update
    finally:
        net.close()
    ref_loss, ref = orp.loss_and_grads(params, feat, label, W, H)
    assert abs(loss - ref_loss) <= 1e-3 * abs(ref_loss) + 1e-4
    # against the backward pass that rounds to BF16 at the kernels' points:
    # what remains is FP32-vs-FP64 accumulation and rare rounding flips
    emu = orp.grads_emulated(params, feat, label, W, H, bf16=True)
    k = 0
    for ci, co in orp.LAYERS:
        for n in (co * ci * 9, co):
            a, b = g[k:k + n], emu[k:k + n]
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
            assert rel <= 1e-2, (k, n, rel)
            # and the plain float64 gradient points the same way
            c = ref[k:k + n]
            assert a @ c / (np.linalg.norm(a) * np.linalg.norm(c)) > 0.99
            k += n


def test_training_reduces_loss():
    import torch
    W, H = 256, 16
    params = sg.net_params_he(31)
    feat = sg.bf16_features_synthetic(32, W, H)
    # a learnable rule: label = feature channel 0 > 0
    label = (feat[:, 0] > 0).astype(np.float32)
    net = capi.Net(params)
    try:
        f, y = _t(feat, torch.bfloat16), _t(label)
        losses = [capi.rt_net_train_step(net.handle, f, y, W, H, 1e-2) for _ in range(40)]
        capi.rt_net_status(net.handle)
        assert not np.array_equal(net.params(), params)
    finally:
        net.close()
    assert losses[-1] < 0.5 * losses[0], losses[::8]


def _full_and_reproj(s, params, threshold):
    import torch
    g = capi.GpuScene(s)
    net = capi.Net(params) if params is not None else None
    try:
        full = g.render()["rgb"]
        L = torch.empty((s.H, s.W, 3), dtype=torch.float32, device="cuda")
        R = torch.empty((s.H, s.W, 3), dtype=torch.float32, device="cuda")
        n = torch.zeros(1, dtype=torch.int32, device="cuda")
        capi.rt_render_stereo_reproj(g.handle, s.camera, s.eye_sep, s.convergence, s.W, s.H,
                                     s.max_depth, net.handle if net else None, threshold, L, R, n)
        capi.rt_sync_status(g.handle)
        if net:
            capi.rt_net_status(net.handle)
        return full, L, R, int(n.item())
    finally:
        g.close()
        if net:
            net.close()


def test_reprojection_with_everything_retraced_equals_full_trace():
    import torch
    s = sg.config_small(1, W=200, H=120)
    params = np.zeros(sg.NET_PARAMS, np.float32)
    params[-1] = 20.0                                     # p = sigmoid(20) ~ 1 everywhere
    full, L, R, n = _full_and_reproj(s, params, 0.5)
    assert n == s.W * s.H
    assert torch.equal(L, full[0]) and torch.equal(R, full[1])


def test_reprojection_holes_only_is_close_to_full_trace():
    import torch
    s = sg.config_small(2, W=320, H=240)
    full, L, R, n = _full_and_reproj(s, None, 0.5)
    assert torch.equal(L, full[0])
    mse = torch.mean((R - full[1]) ** 2).item()
    psnr = 10 * np.log10(1.0 / max(mse, 1e-12))
    assert 0 < n < 0.1 * s.W * s.H and psnr > 25, (n, psnr)


def test_training_pair_labels_cover_holes():
    import torch
    s = sg.config_small(3, W=160, H=96)
    g = capi.GpuScene(s)
    try:
        P = s.W * s.H
        L = torch.empty((s.H, s.W, 3), dtype=torch.float32, device="cuda")
        R = torch.empty_like(L)
        f16 = torch.empty((P, 16), dtype=torch.bfloat16, device="cuda")
        lab = torch.empty(P, dtype=torch.float32, device="cuda")
        capi.rt_reproj_training_pair(g.handle, s.camera, s.eye_sep, s.convergence, s.W, s.H,
                                     s.max_depth, L, R, f16, lab, 1e-2)
        capi.rt_sync_status(g.handle)
        full = g.render()["rgb"]
        assert torch.equal(L, full[0]) and torch.equal(R, full[1])
        holes = (f16.float().abs().sum(dim=1) == 0)
        assert bool((lab[holes] == 1).all())
        assert 0.0 < lab.mean().item() < 0.5
    finally:
        g.close()


# ------------------------------------------------------------------- FP8
FP8_SCALES = (16.0, 16.0, 16.0)


@pytest.mark.parametrize("W,H", [(300, 7), (1, 3), (333, 20)])
def test_fp8_forward_matches_fp8_oracle(W, H):
    """E4M3 activations and weights on kind::f8f6f4 against the float64
    oracle that rounds to E4M3 at the same points; what remains is FP32 vs
    FP64 accumulation, which can move a value across an E4M3 rounding
    boundary (one E4M3 step, 1/16 relative) now and then."""
    import torch
    params = sg.net_params_he(11)
    rng = np.random.default_rng(5)
    params[orp.OFF_B[0]:orp.OFF_B[0] + 32] = rng.normal(0, 0.1, 32)
    params[orp.OFF_B[3]] = -0.5
    feat = sg.bf16_features_synthetic(12, W, H)
    net = capi.Net(params)
    try:
        prob = torch.empty(W * H, dtype=torch.float32, device="cuda")
        f = _t(feat, torch.bfloat16)
        capi.rt_net_forward(net.handle, f, W, H, prob)
        bf16 = prob.clone()
        capi.rt_net_set_fp8(net.handle, FP8_SCALES)
        capi.rt_net_forward(net.handle, f, W, H, prob)
        got = prob.cpu().numpy().reshape(H, W)
        capi.rt_net_set_fp8(net.handle, None)                 # back to BF16, bit for bit
        capi.rt_net_forward(net.handle, f, W, H, prob)
        capi.rt_net_status(net.handle)
        assert torch.equal(prob, bf16)
    finally:
        net.close()
    ref = orp.forward_fp8(params, feat, W, H, FP8_SCALES)
    err = np.abs(got - ref)
    assert err.max() <= 3e-2 and err.mean() <= 1e-3 and (err <= 1e-3).mean() >= 0.98, (err.max(), err.mean())
    # and its distance from the unrounded float64 network (reported, loose bound)
    f64 = orp.forward(params, feat, W, H, bf16=False)
    assert np.abs(got - f64).mean() < 0.02


def test_fp8_scales_rejected_unless_powers_of_two():
    params = sg.net_params_he(3)
    net = capi.Net(params)
    try:
        for bad in ((3.0, 16.0, 16.0), (0.0, 1.0, 1.0), (2.0 ** 40, 1.0, 1.0)):
            with pytest.raises(capi.RtError):
                capi.rt_net_set_fp8(net.handle, bad)
    finally:
        net.close()


def test_activation_amax_matches_bf16_oracle_activations():
    import torch
    W, H = 64, 9
    params = sg.net_params_he(21)
    feat = sg.bf16_features_synthetic(22, W, H)
    net = capi.Net(params)
    try:
        amax = capi.rt_net_activation_amax(net.handle, _t(feat, torch.bfloat16), W, H)
    finally:
        net.close()
    # the oracle's BF16-emulated hidden activations, layer by layer
    import torch.nn.functional as F
    x = torch.tensor(np.asarray(feat, np.float64)[:, :orp.IN_CH].reshape(H, W, orp.IN_CH)).permute(2, 0, 1)[None]
    x = orp._bf16(x)
    want = []
    for w, b in orp.unpack(params)[:3]:
        x = orp._bf16(torch.relu(F.conv2d(x, orp._bf16(torch.tensor(w)), torch.tensor(b), padding=1)))
        want.append(float(x.max()))
    assert np.allclose(amax, want, rtol=2e-2), (amax, want)


def test_fp8_calibration_picks_power_of_two_scales_from_two_maps():
    """rt_net_calibrate_fp8 takes each hidden activation's maximum over all
    the maps it is given and the largest power of two keeping it <= 448; the
    network then runs in FP8 exactly as after rt_net_set_fp8 with them."""
    import torch
    W, H = 64, 9
    params = sg.net_params_he(21)
    fa = _t(sg.bf16_features_synthetic(22, W, H), torch.bfloat16)
    fb = _t(sg.bf16_features_synthetic(23, W, H) * 3.0, torch.bfloat16)
    net = capi.Net(params)
    try:
        a1 = capi.rt_net_activation_amax(net.handle, fa, W, H)
        a2 = capi.rt_net_activation_amax(net.handle, fb, W, H)
        amax, scales = capi.rt_net_calibrate_fp8(net.handle, [fa, fb], W, H)
        prob = torch.empty(W * H, dtype=torch.float32, device="cuda")
        capi.rt_net_forward(net.handle, fa, W, H, prob)
        got = prob.clone()
        capi.rt_net_set_fp8(net.handle, scales)
        capi.rt_net_forward(net.handle, fa, W, H, prob)
        capi.rt_net_status(net.handle)
        assert torch.equal(prob, got)
    finally:
        net.close()
    assert np.array_equal(amax, np.maximum(a1, a2))
    assert np.array_equal(scales, orp.pow2_scale(amax.astype(np.float64)).astype(np.float32))
    assert (scales * amax <= 448).all() and (2 * scales * amax > 448).all()


def test_checkpoint_resumes_training_bit_for_bit(tmp_path):
    """Training is deterministic (weight gradients reduced in a fixed order),
    and a checkpoint holds the parameters, both Adam moments and the step:
    3 steps, save, 3 more steps equals 3 steps, save, load into a new network,
    3 more steps, bit for bit; the file's CRC catches a flipped byte."""
    import torch
    W, H = 300, 40
    f = _t(sg.bf16_features_synthetic(61, W, H), torch.bfloat16)
    y = _t((np.random.default_rng(62).random(W * H) < 0.3).astype(np.float32))
    path = str(tmp_path / "net.ckpt")
    a = capi.Net(sg.net_params_he(63))
    try:
        for _ in range(3):
            capi.rt_net_train_step(a.handle, f, y, W, H, 1e-2, want_loss=False)
        capi.rt_net_save(a.handle, path)
        for _ in range(3):
            capi.rt_net_train_step(a.handle, f, y, W, H, 1e-2, want_loss=False)
        want = a.params()
    finally:
        a.close()
    b = capi.rt_net_load(path)
    try:
        for _ in range(3):
            capi.rt_net_train_step(b, f, y, W, H, 1e-2, want_loss=False)
        capi.rt_net_status(b)
        got = capi.rt_net_get_params(b)
    finally:
        capi.rt_net_destroy(b)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    data = bytearray(open(path, "rb").read())
    data[100] ^= 0x10
    bad = str(tmp_path / "bad.ckpt")
    open(bad, "wb").write(bytes(data))
    with pytest.raises(capi.RtError):
        capi.rt_net_load(bad)


def test_reprojection_with_fp8_network_runs_and_matches_bf16_closely():
    import torch
    from paper_1702_01530_gb300 import train_reproj as tr
    s = sg.config_small(4, W=320, H=240)
    params, thr = tr.load_weights()
    g = capi.GpuScene(s)
    net = capi.Net(params)
    try:
        full = g.render()["rgb"]
        outs = {}
        for mode in ("bf16", "fp8"):
            if mode == "fp8":
                capi.rt_net_set_fp8(net.handle, FP8_SCALES)
            L = torch.empty((s.H, s.W, 3), dtype=torch.float32, device="cuda")
            R = torch.empty_like(L)
            n = torch.zeros(1, dtype=torch.int32, device="cuda")
            capi.rt_render_stereo_reproj(g.handle, s.camera, s.eye_sep, s.convergence, s.W, s.H,
                                         s.max_depth, net.handle, thr, L, R, n)
            capi.rt_sync_status(g.handle)
            capi.rt_net_status(net.handle)
            outs[mode] = (L, R, int(n.item()))
        assert torch.equal(outs["fp8"][0], full[0])
        p = {m: tr.psnr(outs[m][1], full[1]) for m in outs}
        assert p["fp8"] > p["bf16"] - 1.0, p
        assert abs(outs["fp8"][2] - outs["bf16"][2]) <= 0.2 * max(outs["bf16"][2], 100)
    finally:
        net.close()
        g.close()


# ------------------------------------------- persistent multi-tile path
# The convolution kernel is persistent: a grid of (SMs x CTAs per SM) walks
# the tiles of 128 pixels x 4 rows, each CTA through a ring of 3 halo
# buffers and 2 TMEM accumulator sets. These sizes give every CTA of every
# layer (2 CTAs per SM for the 16-channel layers, 1 for the 32-channel ones)
# at least 4 tiles, so the ring wraps, both accumulator sets are reused and
# the barrier parities flip; the widths leave a ragged last column tile.
MULTI = [(1920, 544), (1000, 620)]


def _tiles_per_cta(W, H, ctas_per_sm):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tiles = -(-W // 128) * -(-H // 4)
    return tiles / (sms * ctas_per_sm)


@pytest.mark.parametrize("W,H", MULTI)
def test_network_forward_multi_tile_per_cta(W, H):
    import torch
    assert _tiles_per_cta(W, H, 2) >= 4
    params = sg.net_params_he(41)
    rng = np.random.default_rng(42)
    params[orp.OFF_B[0]:orp.OFF_B[0] + 32] = rng.normal(0, 0.1, 32)
    params[orp.OFF_B[3]] = -0.5
    feat = sg.bf16_features_synthetic(43, W, H)
    net = capi.Net(params)
    try:
        prob = torch.empty(W * H, dtype=torch.float32, device="cuda")
        f = _t(feat, torch.bfloat16)
        capi.rt_net_forward(net.handle, f, W, H, prob)
        got = prob.cpu().numpy().reshape(H, W)
        capi.rt_net_set_fp8(net.handle, FP8_SCALES)
        capi.rt_net_forward(net.handle, f, W, H, prob)
        got8 = prob.cpu().numpy().reshape(H, W)
        capi.rt_net_status(net.handle)
    finally:
        net.close()
    ref = orp.forward(params, feat, W, H, bf16=True)
    err = np.abs(got - ref)
    assert err.max() <= 5e-3 and err.mean() <= 2e-4, (err.max(), err.mean())
    ref8 = orp.forward_fp8(params, feat, W, H, FP8_SCALES)
    err8 = np.abs(got8 - ref8)
    assert err8.max() <= 3e-2 and err8.mean() <= 1e-3 and (err8 <= 1e-3).mean() >= 0.98, \
        (err8.max(), err8.mean())
    # every tile row of the last column and the last tile row are covered
    assert ref.std() > 1e-3 and np.isfinite(got).all()


@pytest.mark.parametrize("W,H", MULTI[:1])
def test_gradients_multi_tile_per_cta(W, H):
    import torch
    assert _tiles_per_cta(W, H, 2) >= 4
    params = sg.net_params_he(51)
    params[orp.OFF_B[3]] = 0.2
    feat = sg.bf16_features_synthetic(52, W, H)
    label = (np.random.default_rng(53).random(W * H) < 0.3).astype(np.float32)
    net = capi.Net(params)
    try:
        grads = torch.zeros(capi.RT_NET_PARAMS, dtype=torch.float32, device="cuda")
        capi.rt_net_train_step(net.handle, _t(feat, torch.bfloat16), _t(label), W, H, 0.0,
                               grads=grads)
        capi.rt_net_status(net.handle)
        g = grads.cpu().numpy().astype(np.float64)
    finally:
        net.close()
    emu = orp.grads_emulated(params, feat, label, W, H, bf16=True)
    k = 0
    for ci, co in orp.LAYERS:
        for n in (co * ci * 9, co):
            a, b = g[k:k + n], emu[k:k + n]
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
            assert rel <= 1e-2, (k, n, rel)
            k += n


# ---------------------------------------------- mixed retrace mask (A9)
def test_reprojection_mixed_mask_matches_oracle():
    """Trained weights at threshold 0.1 on a 320x240 small scene: the right
    pixels retraced are the holes, the pixels showing a reflective surface
    and the pixels whose oracle probability (on the GPU's own features)
    exceeds the threshold; retraced pixels equal the full trace, the others
    the oracle's warped left colour. Pixels whose probability lies within
    5e-3 of the threshold may go either way."""
    import torch
    from paper_1702_01530_gb300 import train_reproj as tr
    s = sg.config_small(7, W=320, H=240)
    params, _ = tr.load_weights()
    thr = 0.1
    W, H, P = s.W, s.H, s.W * s.H
    g = capi.GpuScene(s)
    net = capi.Net(params)
    try:
        full = g.render(aux=True)
        depth_L = full["depth"][0].cpu().numpy()
        hit_L = full["hit_id"][0].cpu().numpy().view(np.uint32).reshape(P)
        fL, fR = full["rgb"][0], full["rgb"][1]
        L = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
        R = torch.empty_like(L)
        f16 = torch.empty((P, 16), dtype=torch.bfloat16, device="cuda")
        lab = torch.empty(P, dtype=torch.float32, device="cuda")
        capi.rt_reproj_training_pair(g.handle, s.camera, s.eye_sep, s.convergence, W, H,
                                     s.max_depth, L, R, f16, lab, 1e-2)
        feat = f16.float().cpu().numpy()
        n = torch.zeros(1, dtype=torch.int32, device="cuda")
        capi.rt_render_stereo_reproj(g.handle, s.camera, s.eye_sep, s.convergence, W, H,
                                     s.max_depth, net.handle, thr, L, R, n)
        capi.rt_sync_status(g.handle)
        capi.rt_net_status(net.handle)
        assert torch.equal(L, fL)
        Lh, Rh, fRh = L.cpu().numpy(), R.cpu().numpy(), fR.cpu().numpy()
    finally:
        net.close()
        g.close()
    f_px = capi.focal_px(s.camera, H)
    # reflectivity of each left pixel's surface (ids: spheres first, then triangles)
    refl_of_id = np.concatenate([s.materials["reflectivity"][s.spheres["material"]],
                                 s.materials["reflectivity"][s.triangles["material"]]])
    refl_L = np.where(hit_L == capi.RT_MISS_ID, 0.0, refl_of_id[np.minimum(hit_L, len(refl_of_id) - 1)])
    ofeat, hole, warped, _ = orp.warp(depth_L, np.zeros((P, 3)), np.zeros(P, np.uint32), Lh, W, H,
                                      f_px, s.eye_sep, s.convergence, refl_L.astype(np.float32))
    mirror = ~hole & (ofeat[:, 9] > 0)
    assert np.array_equal(ofeat[:, 9] > 0, feat[:, 9] > 0)             # the GPU's feature agrees
    p = orp.forward(params, feat, W, H, bf16=True).reshape(P)
    near = np.abs(p - thr) < 5e-3
    want = hole | mirror | (p > thr)
    R2, F2, Wp = Rh.reshape(P, 3), fRh.reshape(P, 3), warped.reshape(P, 3).astype(np.float32)
    sel = want & ~near
    assert np.array_equal(R2[sel], F2[sel])                       # retraced = full trace
    keep = ~want & ~near
    assert np.array_equal(R2[keep], Wp[keep])                     # others = warped colour
    assert abs(int(n.item()) - int(want.sum())) <= int(near.sum())
    # a mixed mask: some pixels retraced for p > thr beyond the holes, most kept
    assert (want & ~hole & ~mirror).sum() > 0 and 0 < want.mean() < 0.5, (want.sum(), hole.sum())


def _bf16_bits(x):
    """float32 -> BF16 bit patterns, round to nearest even (finite inputs)."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def test_network_full_size_sampled_matches_oracle():
    """The launch the terrain reprojection times: 8 images of 3840x2160 per
    call, BF16 and FP8. Each output depends on the 9x9 window of inputs
    around it (four 3x3 layers), so the oracle computes sampled pixels from
    crops: tile edges (126-pixel tiles of the chunk-planar layers, 128 of the
    first layer, rows in fours), image borders and random pixels. Features:
    image i tiles a seeded 1024x1024 block with an offset of its own."""
    import torch
    W, H, N, B = 3840, 2160, 8, 1024
    params = sg.net_params_he(51)
    rng = np.random.default_rng(52)
    params[orp.OFF_B[0]:orp.OFF_B[0] + 32] = rng.normal(0, 0.1, 32)
    params[orp.OFF_B[3]] = -0.5
    block = np.zeros((B, B, 16), np.uint16)
    block[..., :orp.IN_CH] = _bf16_bits(np.clip(rng.normal(0, 0.8, (B, B, orp.IN_CH)), -2, 2))
    block_f = (block.astype(np.uint32) << 16).view(np.float32)
    offs = [(int(rng.integers(B)), int(rng.integers(B))) for _ in range(N)]
    yy, xx = np.arange(H)[:, None], np.arange(W)[None, :]
    feat = torch.empty((N, H, W, 16), dtype=torch.bfloat16, device="cuda")
    for i, (oy, ox) in enumerate(offs):
        img = block[(yy + oy) % B, (xx + ox) % B]
        feat[i].copy_(torch.from_numpy(img).view(torch.bfloat16))
    samples = [(0, 0, 0), (1, H - 1, W - 1), (2, 0, W - 1), (3, H - 1, 0)]
    for i in range(N):
        for y in (1, 3, 4, 7, 8, H - 2):
            for x in (1, 125, 126, 127, 128, 251, 252, 253, W - 2):
                if rng.random() < 0.35:
                    samples.append((i, y, x))
    samples += [(int(rng.integers(N)), int(rng.integers(H)), int(rng.integers(W))) for _ in range(40)]
    net = capi.Net(params)
    try:
        prob = torch.empty((N, H, W), dtype=torch.float32, device="cuda")
        capi.rt_net_forward_images(net.handle, feat, N, W, H, prob)
        got16 = prob.cpu().numpy()
        capi.rt_net_set_fp8(net.handle, FP8_SCALES)
        capi.rt_net_forward_images(net.handle, feat, N, W, H, prob)
        got8 = prob.cpu().numpy()
        capi.rt_net_status(net.handle)
    finally:
        net.close()
    e16, e8 = [], []
    for i, y, x in samples:
        y0, y1, x0, x1 = max(0, y - 4), min(H, y + 5), max(0, x - 4), min(W, x + 5)
        oy, ox = offs[i]
        crop = block_f[(np.arange(y0, y1)[:, None] + oy) % B, (np.arange(x0, x1)[None, :] + ox) % B]
        h, w = y1 - y0, x1 - x0
        flat = crop.reshape(h * w, 16).astype(np.float64)
        r16 = orp.forward(params, flat, w, h, bf16=True)[y - y0, x - x0]
        r8 = orp.forward_fp8(params, flat, w, h, FP8_SCALES)[y - y0, x - x0]
        e16.append(abs(got16[i, y, x] - r16))
        e8.append(abs(got8[i, y, x] - r8))
    e16, e8 = np.array(e16), np.array(e8)
    assert len(samples) > 150
    assert e16.max() <= 5e-3 and e16.mean() <= 5e-4, (e16.max(), e16.mean())
    assert e8.max() <= 3e-2 and e8.mean() <= 2e-3, (e8.max(), e8.mean())
    assert np.isfinite(got16).all() and np.isfinite(got8).all() and got16.std() > 1e-3
