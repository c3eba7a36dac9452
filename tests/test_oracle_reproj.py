"""Pins of the reprojection / network oracle (CPU only)."""
import math

import numpy as np
import pytest

from oracle import reproj as orp
from paper_1702_01530_gb300 import scenegen as sg


def _fmix32_int(h):
    h &= 0xFFFFFFFF
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & 0xFFFFFFFF
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & 0xFFFFFFFF
    h ^= h >> 16
    return h


def test_fmix32_matches_integer_definition_and_known_values():
    assert _fmix32_int(0) == 0 and _fmix32_int(1) == 0x514E28B7
    xs = np.array([0, 1, 2, 999, 0xFFFFFFFF, 123456789], np.uint32)
    assert orp.fmix32(xs).tolist() == [_fmix32_int(int(x)) for x in xs]


def _plane(W, H, z):
    P = W * H
    depth = np.full(P, z, np.float32)
    normal = np.tile(np.array([0, 0, 1], np.float32), (P, 1))
    ids = np.arange(P, dtype=np.uint32)
    rgb = np.random.default_rng(0).random((P, 3)).astype(np.float32)
    return depth, normal, ids, rgb


def test_warp_of_fronto_parallel_plane_is_a_uniform_shift():
    # D = f s (1/z - 1/zc) = 100 * 0.1 * (1/2.5 - 1/10) = 3 pixels exactly
    W, H = 40, 6
    depth, normal, ids, rgb = _plane(W, H, 2.5)
    D = orp.disparity32(2.5, 100.0, 0.1, 10.0)
    assert D == np.float32(3.0)
    feat, hole, warped, src = orp.warp(depth, normal, ids, rgb, W, H, 100.0, 0.1, 10.0)
    hole = hole.reshape(H, W)
    assert hole[:, W - 3:].all() and not hole[:, :W - 3].any()     # right edge uncovered
    src = src.reshape(H, W)
    jj, ii = np.mgrid[0:H, 0:W - 3]
    assert np.array_equal(src[:, :W - 3], jj * W + ii + 3)         # x_R = x_L - 3
    f = feat.reshape(H, W, orp.IN_CH)
    assert np.allclose(f[:, :W - 3, 8], 3.0 / 16) and np.allclose(f[:, :W - 3, 0], 0.025)
    assert np.allclose(f[:, :W - 3, 1:4], [0, 0, 1]) and (f[:, W - 3:] == 0).all()
    # misses are sources at infinity: D = -f s / zc = -1 -> they fill column 0.. from the left
    depth_m = np.full(W * H, np.inf, np.float32)
    _, hole_m, _, src_m = orp.warp(depth_m, normal, ids, rgb, W, H, 100.0, 0.1, 10.0)
    assert hole_m.reshape(H, W)[:, 0].all() and not hole_m.reshape(H, W)[:, 1:].any()
    assert src_m.reshape(H, W)[0, 1] == 0
    # farther than the convergence plane: the shift goes the other way
    depth2 = np.full(W * H, 40.0, np.float32)                      # D = 10 (0.025 - 0.1) = -0.75
    _, hole2, _, src2 = orp.warp(depth2, normal, ids, rgb, W, H, 100.0, 0.1, 10.0)
    assert hole2.reshape(H, W)[:, 0].all() and not hole2.reshape(H, W)[:, 1:].any()
    assert src2.reshape(H, W)[0, 5] == 4                           # floor(4 + 0.75 + 0.5) = 5


def test_warp_carries_reflectivity_of_the_source_pixel():
    W, H = 40, 6
    depth, normal, ids, rgb = _plane(W, H, 2.5)
    refl = (np.arange(W * H) % 7 / 10.0).astype(np.float32)
    feat, hole, _, src = orp.warp(depth, normal, ids, rgb, W, H, 100.0, 0.1, 10.0, refl)
    ok = ~hole
    assert np.array_equal(feat[ok, 9], refl[src[ok]].astype(np.float64)) and (feat[hole] == 0).all()
    assert (orp.warp(depth, normal, ids, rgb, W, H, 100.0, 0.1, 10.0)[0][:, 9] == 0).all()


def test_warp_z_test_keeps_nearest_then_lowest_index():
    W, H = 8, 1
    depth = np.zeros(8, np.float32)       # depth <= 0: not a source
    # pixels 5 and 6 both land on column 3 with f=100, s=0.1, zc=10:
    # pixel 5 at D=2 (z=1/(0.2+0.1)), pixel 6 at D=3 (z=2.5)
    z5 = np.float32(1.0 / 0.3)
    depth[5], depth[6] = z5, 2.5
    d5 = orp.disparity32(z5, 100.0, 0.1, 10.0)
    assert math.floor(5 - d5 + 0.5) == 3
    normal = np.zeros((8, 3), np.float32)
    ids = np.arange(8, dtype=np.uint32)
    rgb = np.zeros((8, 3), np.float32)
    _, hole, _, src = orp.warp(depth, normal, ids, rgb, W, H, 100.0, 0.1, 10.0)
    assert src[3] == 6                    # z = 2.5 is nearer than 3.33
    depth[5] = 2.5                        # now equal depth: lands on 2.. move both to one target
    depth[4] = 2.5                        # pixel 4 -> column 1, pixel 5 -> 2, pixel 6 -> 3
    _, _, _, src = orp.warp(depth, normal, ids, rgb, W, H, 100.0, 0.1, 10.0)
    assert src[1:4].tolist() == [4, 5, 6] and hole.sum() == 7


def test_labels_definition():
    hole = np.array([1, 0, 0, 0], bool)
    w = np.zeros((4, 3))
    f = np.array([[0, 0, 0], [0.005, 0, 0], [0, 0.0101, 0], [0, 0, 0]])
    assert orp.labels(hole, w, f, 1e-2).tolist() == [1, 0, 1, 0]


def _conv_loops(x, w, b):
    """Explicit 3x3 zero-padded cross-correlation (independent of PyTorch)."""
    C, H, W = x.shape
    co = w.shape[0]
    out = np.zeros((co, H, W))
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    for o in range(co):
        for y in range(H):
            for xx in range(W):
                out[o, y, xx] = b[o] + np.sum(w[o] * xp[:, y:y + 3, xx:xx + 3])
    return out


def test_network_forward_matches_explicit_loops():
    W, H = 5, 4
    params = sg.net_params_he(3).astype(np.float64)
    params[params.size - 1] = 0.3
    feat = sg.bf16_features_synthetic(4, W, H)
    x = feat[:, :orp.IN_CH].reshape(H, W, orp.IN_CH).transpose(2, 0, 1).astype(np.float64)
    for li, (w, b) in enumerate(orp.unpack(params)):
        x = _conv_loops(x, w, b)
        if li < 3:
            x = np.maximum(x, 0)
    ref = 1 / (1 + np.exp(-x[0]))
    assert np.allclose(orp.forward(params, feat, W, H, bf16=False), ref, atol=1e-12)
    assert np.abs(orp.forward(params, feat, W, H, bf16=True) - ref).max() < 2e-2


def test_network_constant_output_and_bce_closed_form():
    W, H = 6, 3
    params = np.zeros(sg.NET_PARAMS)
    params[-1] = 2.0
    feat = sg.bf16_features_synthetic(5, W, H)
    assert np.allclose(orp.forward(params, feat, W, H), 1 / (1 + math.exp(-2.0)))
    y = (np.arange(W * H) % 3 == 0).astype(np.float64)
    s = 1 / (1 + math.exp(-2.0))
    loss, g = orp.loss_and_grads(params, feat, y, W, H)
    assert abs(loss - (-(y * math.log(s) + (1 - y) * math.log(1 - s)).mean())) < 1e-12
    assert abs(g[-1] - (s - y).mean()) < 1e-12          # d loss / d b4 = mean(p - y)


def test_network_gradient_matches_central_differences():
    W, H = 5, 4
    params = sg.net_params_he(7).astype(np.float64)
    params += 0.01 * np.random.default_rng(1).standard_normal(params.size)
    feat = sg.bf16_features_synthetic(8, W, H)
    y = (np.random.default_rng(2).random(W * H) < 0.3).astype(np.float64)
    _, g = orp.loss_and_grads(params, feat, y, W, H)
    rng = np.random.default_rng(3)
    B, Wo = orp.OFF_B, orp.OFF_W
    idx = np.concatenate([rng.choice(B[0], 6, replace=False),
                          [B[0] + 8, Wo[1] + 5, B[2] - 1, Wo[3] + 7, B[3]]])
    h = 1e-6
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        fd = (orp.loss_and_grads(pp, feat, y, W, H)[0] - orp.loss_and_grads(pm, feat, y, W, H)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_emulated_backward_equals_autograd_without_rounding():
    W, H = 6, 5
    params = sg.net_params_he(9).astype(np.float64)
    params[orp.OFF_B[0]:orp.OFF_B[0] + 32] = 0.05
    feat = sg.bf16_features_synthetic(10, W, H)
    y = (np.random.default_rng(4).random(W * H) < 0.4).astype(np.float64)
    _, g = orp.loss_and_grads(params, feat, y, W, H)
    ge = orp.grads_emulated(params, feat, y, W, H, bf16=False)
    assert np.abs(ge - g).max() <= 1e-12 * max(1.0, np.abs(g).max())
    gb = orp.grads_emulated(params, feat, y, W, H, bf16=True)
    cos = gb @ g / (np.linalg.norm(gb) * np.linalg.norm(g))
    assert cos > 0.99


def test_generators_for_reprojection():
    d, n, ids, rgb, refl = sg.gbuffer_synthetic(1, 30, 20)
    assert set(np.unique(refl[~np.isinf(d)]).tolist()) <= set(np.float32([0.0, 0.5, 0.7]).tolist())
    assert (refl[np.isinf(d)] == 0).all()
    assert np.isinf(d).mean() == pytest.approx(0.2, abs=0.06)
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-6)
    assert (ids[np.isinf(d)] == 0xFFFFFFFF).all() and (ids[~np.isinf(d)] < 1000).all()
    f = sg.bf16_features_synthetic(2, 10, 10)
    import torch
    t = torch.tensor(f)
    assert torch.equal(t.to(torch.bfloat16).to(torch.float32), t)
    p = sg.net_params_he(0)
    assert p.size == sg.NET_PARAMS == orp.N_PARAMS == 21697 and p[orp.OFF_B[0]:orp.OFF_B[0] + 32].max() == 0


def test_composite_oracle_definitions():
    from oracle import post
    L = np.zeros((2, 3, 3), np.float32)
    R = np.ones((2, 3, 3), np.float32)
    L[..., 0] = 0.25
    c = post.composite(L, R, 0)
    assert (c[..., 0] == 0.25).all() and (c[..., 1:] == 1).all()
    g = post.composite(L, R, 1)
    assert np.allclose(g[..., 0], 0.299 * 0.25) and np.allclose(g[..., 1:], 1.0, atol=1e-6)
    sbs = post.composite(L, R, 2)
    assert sbs.shape == (2, 6, 3) and (sbs[:, :3] == L).all() and (sbs[:, 3:] == R).all()


# ------------------------------------------------------------------- FP8
def _e4m3_table():
    """Every finite E4M3 value from the bit layout: sign, 4 exponent bits
    (bias 7), 3 mantissa bits; exponent 0 is subnormal (M * 2^-9); the
    pattern S.1111.111 is NaN."""
    vals = []
    for b in range(256):
        sgn, E, M = b >> 7, (b >> 3) & 15, b & 7
        if E == 15 and M == 7:
            continue
        v = M * 2.0 ** -9 if E == 0 else (1 + M / 8) * 2.0 ** (E - 7)
        vals.append((-v if sgn else v, M))
    return vals


def test_e4m3_table_limits():
    t = sorted(v for v, _ in _e4m3_table())
    assert max(t) == 448.0 and min(t) == -448.0
    assert min(v for v in t if v > 0) == 2.0 ** -9
    assert np.array_equal(orp.e4m3(np.array(t)), np.array(t))      # representable values are fixed


def test_e4m3_rounding_matches_brute_force_nearest_even():
    table = _e4m3_table()
    vals = np.array([v for v, _ in table])
    mant = np.array([m for _, m in table])
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-500, 500, 400),
                        np.exp2(rng.uniform(-12, 9.5, 400)) * rng.choice([-1, 1], 400),
                        (vals[:-1] + vals[1:]) / 2.0])                # exact ties
    got = orp.e4m3(x)
    for xi, gi in zip(x, got):
        if abs(xi) >= 448.0:
            assert gi == np.copysign(448.0, xi)
            continue
        d = np.abs(vals - xi)
        cand = np.flatnonzero(d == d.min())
        if len(cand) > 1:                                  # tie: the even mantissa wins
            cand = [c for c in cand if mant[c] % 2 == 0]
        assert gi == vals[cand[0]] or (gi == 0 and vals[cand[0]] == 0), (xi, gi, vals[cand])


def test_pow2_scale():
    s = orp.pow2_scale(np.array([1.0, 448.0, 449.0, 3.5, 0.0, 1e-3]))
    assert s.tolist() == [256.0, 1.0, 0.5, 128.0, 1.0, 262144.0]
    a = np.random.default_rng(4).uniform(1e-3, 1e3, 100)
    sc = orp.pow2_scale(a)
    assert (a * sc <= 448.0).all() and (a * sc * 2 > 448.0).all()


def test_fp8_forward_identity_network_closed_form():
    # layer 1 copies feature 0 to channel 0, layers 2 and 3 pass channel 0
    # through, layer 4 reads it with bias b: p = sigmoid(x0 + b) exactly when
    # x0 is representable after scaling, whatever the scales
    W, H = 11, 7
    params = np.zeros(sum(ci * co * 9 + co for ci, co in orp.LAYERS), np.float32)
    k = 0
    for li, (ci, co) in enumerate(orp.LAYERS):
        w = np.zeros((co, ci, 3, 3), np.float32)
        w[0, 0, 1, 1] = 1.0
        params[k:k + w.size] = w.ravel()
        k += w.size
        if li == 3:
            params[k] = -0.75
        k += co
    rng = np.random.default_rng(5)
    feat = np.zeros((W * H, 16), np.float32)
    feat[:, 0] = rng.integers(0, 16, W * H) / 8.0
    feat[:, 1:orp.IN_CH] = rng.uniform(-1, 1, (W * H, orp.IN_CH - 1))
    for scales in ((16.0, 16.0, 16.0), (1.0, 64.0, 0.5)):
        p = orp.forward_fp8(params, feat, W, H, scales)
        want = 1.0 / (1.0 + np.exp(-(feat[:, 0].astype(np.float64).reshape(H, W) - 0.75)))
        assert np.allclose(p, want, rtol=0, atol=1e-15)
    # dropping the weight scale (a plausible slip) would multiply x0 by 256
    assert orp.weight_scales_fp8(params)[0][0] == 256.0


def test_fp8_forward_close_to_float64_network():
    W, H = 40, 12
    params = sg.net_params_he(41)
    feat = sg.bf16_features_synthetic(42, W, H)
    ref = orp.forward(params, feat, W, H, bf16=False)
    x = orp.forward(params, feat, W, H, bf16=True)            # hidden activations' range
    p8 = orp.forward_fp8(params, feat, W, H, (8.0, 8.0, 8.0))
    assert np.abs(p8 - ref).max() < 0.1 and np.abs(p8 - ref).mean() < 0.02
    assert np.abs(x - ref).max() < np.abs(p8 - ref).max()     # FP8 loses more than BF16


# ---------------------------------- BF16 rounding points, pinned exactly
# Independent restatements (no PyTorch convolution or autograd) of the
# network with BF16 rounding where the tensor-core kernels round: inputs,
# weights and hidden activations in the forward pass; the (p - y) map fed
# to the layer-4 data gradient (the layer-4 weight gradient takes p - y
# unrounded) and every data gradient after its ReLU mask in the backward
# pass. Random values carry ~50 significant bits, so each rounding moves
# results by ~2^-9 relative: dropping or moving one rounding point fails the
# 1e-9 comparisons below by many orders of magnitude.
def _rne_bf16(x):
    """Round to 8 significant bits, ties to even (BF16 in its normal range)."""
    m, e = np.frexp(np.asarray(x, np.float64))
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def _pad(a):
    C, H, W = a.shape
    ap = np.zeros((C, H + 2, W + 2))
    ap[:, 1:-1, 1:-1] = a
    return ap


def _conv_wgrad(a, dz):
    """dW[o, c, ky, kx] = sum_{y, x} dz[o, y, x] a_pad[c, y + ky, x + kx]."""
    C, H, W = a.shape
    ap = _pad(a)
    dW = np.zeros((dz.shape[0], C, 3, 3))
    for ky in range(3):
        for kx in range(3):
            dW[:, :, ky, kx] = np.einsum("oyx,cyx->oc", dz, ap[:, ky:ky + H, kx:kx + W])
    return dW


def _conv_dgrad(dz, w, H, W):
    """Data gradient of a 3x3 zero-padded cross-correlation: every output
    dz[o, y, x] sends w[o, c, ky, kx] dz[o, y, x] back to input (c, y+ky-1,
    x+kx-1)."""
    dap = np.zeros((w.shape[1], H + 2, W + 2))
    for ky in range(3):
        for kx in range(3):
            dap[:, ky:ky + H, kx:kx + W] += np.einsum("oc,oyx->cyx", w[:, :, ky, kx], dz)
    return dap[:, 1:-1, 1:-1]


def _net_loops_bf16(params, feat, label, W, H):
    """Probability map and mean-BCE gradient with BF16 rounding points."""
    layers = orp.unpack(np.asarray(params, np.float64))
    a = [_rne_bf16(np.asarray(feat, np.float64)[:, :orp.IN_CH].reshape(H, W, orp.IN_CH).transpose(2, 0, 1))]
    for li in range(3):
        w, b = layers[li]
        a.append(_rne_bf16(np.maximum(_conv_loops(a[-1], _rne_bf16(w), b), 0.0)))
    w4, b4 = layers[3]
    q = 1.0 / (1.0 + np.exp(-_conv_loops(a[3], _rne_bf16(w4), b4)))
    P = W * H
    g = q - np.asarray(label, np.float64).reshape(1, H, W)
    grads = [None] * 4
    dz_w, dz_in = g, _rne_bf16(g)            # layer 4: weight gradient unrounded
    for li in (3, 2, 1, 0):
        w, _ = layers[li]
        grads[li] = (_conv_wgrad(a[li], dz_w) / P, dz_w.sum(axis=(1, 2)) / P)
        if li > 0:
            da = _conv_dgrad(dz_in, _rne_bf16(w), H, W)
            dz_w = dz_in = _rne_bf16(da * (a[li] > 0))
    flat = np.concatenate([np.concatenate([dw.reshape(-1), db]) for dw, db in grads])
    return q[0], flat


def _bf16_case():
    W, H = 7, 5
    params = sg.net_params_he(15).astype(np.float64)
    params += 0.01 * np.random.default_rng(16).standard_normal(params.size)
    feat = np.random.default_rng(17).random((W * H, 16))        # not BF16 values
    y = (np.random.default_rng(18).random(W * H) < 0.4).astype(np.float64)
    return params, feat, y, W, H


def check_forward_bf16(mod):
    params, feat, _, W, H = _bf16_case()
    q, _ = _net_loops_bf16(params, feat, np.zeros(W * H), W, H)
    got = mod.forward(params, feat, W, H, bf16=True)
    assert np.abs(got - q).max() <= 1e-9, np.abs(got - q).max()


def check_grads_bf16(mod):
    params, feat, y, W, H = _bf16_case()
    _, g = _net_loops_bf16(params, feat, y, W, H)
    got = mod.grads_emulated(params, feat, y, W, H, bf16=True)
    k = 0
    for ci, co in orp.LAYERS:
        for n in (co * ci * 9, co):
            a, b = got[k:k + n], g[k:k + n]
            assert np.abs(a - b).max() <= 1e-9 * max(1e-3, np.abs(b).max()), (k, n, np.abs(a - b).max())
            k += n


def test_forward_bf16_rounding_points_match_explicit_loops():
    check_forward_bf16(orp)
    # the rounding matters at this size: the unrounded network is far away
    params, feat, _, W, H = _bf16_case()
    q, _ = _net_loops_bf16(params, feat, np.zeros(W * H), W, H)
    assert np.abs(orp.forward(params, feat, W, H, bf16=False) - q).max() > 1e-5


def test_emulated_backward_bf16_rounding_points_match_explicit_loops():
    check_grads_bf16(orp)
    params, feat, y, W, H = _bf16_case()
    _, g = _net_loops_bf16(params, feat, y, W, H)
    plain = orp.grads_emulated(params, feat, y, W, H, bf16=False)
    assert np.abs(plain - g).max() > 1e-6


def test_rne_bf16_helper_against_hand_values():
    # 1 + 2^-8 is the tie between 1 and 1 + 2^-7: even mantissa -> 1
    assert _rne_bf16(1.0 + 2.0 ** -8) == 1.0
    assert _rne_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6     # tie -> even (...10)
    assert _rne_bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert _rne_bf16(-3.0) == -3.0 and _rne_bf16(0.0) == 0.0
    assert _rne_bf16(255.5) == 256.0 and _rne_bf16(2.0 ** 130 * 1.3) == 2.0 ** 130 * (166 / 128)
