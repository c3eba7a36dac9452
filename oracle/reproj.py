"""Oracle of the learned right-eye reprojection -- TEST INFRASTRUCTURE.

Only tests, smoke() and bench.py's CPU leg may import this module. Plain
definitions in numpy (and PyTorch CPU float64 for the network):

* forward warp: a left pixel (i, j) at view depth z lands on column
  floor(i - D + 0.5) of row j with D = f_px * s * (1/z - 1/zc); the target
  keeps the nearest z, equal z the lower left index; a miss (z = +inf) is a
  source at infinity (D = -f_px s / zc). The disparity and the
  target column are evaluated in float32 with the same operations as the
  kernel (one IEEE operation at a time), because they decide an integer.
* features of a right pixel: min(z/100, 1), normal, hash(id) =
  (fmix32(id) >> 8) 2^-24 (MurmurHash3 finaliser), left RGB, D/16, the
  reflectivity of the left pixel's surface; zeros on a hole. Labels: hole
  or max_c |warped - full| > threshold.
* network: 3x3 convolutions 10 -> 32 -> 32 -> 32 -> 1 with zero padding 1,
  ReLU, sigmoid; mean binary cross-entropy; gradients by autograd in float64.
  `forward(..., bf16=True)` rounds inputs, weights and hidden activations to
  BF16 where the tensor-core kernels do, so the two can be compared closely.
* FP8 inference (`forward_fp8`): the first layer as in the BF16 network; its
  output and every later hidden activation is stored as OCP FP8 E4M3 of the
  activation times a per-tensor power-of-two scale; layers 2-4 use E4M3
  weights times a per-output-channel power-of-two scale (`weight_scales_fp8`),
  undone (exactly) before the bias. E4M3 (`e4m3`): sign, 4 exponent bits
  with bias 7, 3 mantissa bits, subnormals below 2^-6, largest finite 448,
  no infinities; conversion rounds to nearest, ties to even mantissa, and
  saturates to +-448.
"""
from __future__ import annotations

import numpy as np

Z_FAR = 100.0
DISP_SCALE = 1.0 / 16.0
LAYERS = ((10, 32), (32, 32), (32, 32), (32, 1))
IN_CH = LAYERS[0][0]              # feature channels the network reads
# offsets of each layer's weights and biases in the parameter vector
OFF_W, OFF_B = [], []
_k = 0
for _ci, _co in LAYERS:
    OFF_W.append(_k)
    OFF_B.append(_k + _co * _ci * 9)
    _k += _co * _ci * 9 + _co
N_PARAMS = _k


def fmix32(h):
    h = np.asarray(h, dtype=np.uint64) & np.uint64(0xFFFFFFFF)
    m = np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(16)
    h = (h * np.uint64(0x85EBCA6B)) & m
    h ^= h >> np.uint64(13)
    h = (h * np.uint64(0xC2B2AE35)) & m
    h ^= h >> np.uint64(16)
    return h.astype(np.uint32)


def disparity32(z, f_px, eye_sep, convergence):
    f32 = np.float32
    fs = f32(f_px) * f32(eye_sep)
    inv_zc = f32(1.0) / f32(convergence)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        return fs * (f32(1.0) / np.asarray(z, np.float32) - inv_zc)


def warp(depth, normal, ids, rgb, W, H, f_px, eye_sep, convergence, refl=None):
    """Returns features (P, 10) float64, hole (P,) bool, warped RGB (P, 3),
    source index (P,) int64 (-1 on a hole). refl: reflectivity of each left
    pixel's surface (None: zeros)."""
    P = W * H
    z = np.asarray(depth, np.float32).reshape(P)
    with np.errstate(invalid="ignore"):
        valid = z > 0                              # +inf (a miss) included, NaN excluded
    D = disparity32(z, f_px, eye_sep, convergence)
    i = (np.arange(P) % W).astype(np.float32)
    j = np.arange(P) // W
    with np.errstate(invalid="ignore"):
        c = np.floor((i - D) + np.float32(0.5))
        ok = valid & (c >= 0) & (c < W)
    srcs = np.nonzero(ok)[0]
    tgt = j[srcs] * W + c[srcs].astype(np.int64)
    order = np.lexsort((srcs, z[srcs], tgt))           # by target, then z, then index
    tgt_s, src_s = tgt[order], srcs[order]
    first = np.ones(len(tgt_s), bool)
    first[1:] = tgt_s[1:] != tgt_s[:-1]
    source = np.full(P, -1, np.int64)
    source[tgt_s[first]] = src_s[first]
    hole = source < 0
    q = np.where(hole, 0, source)
    feat = np.zeros((P, IN_CH), np.float64)
    zq = z[q].astype(np.float64)
    with np.errstate(invalid="ignore"):
        feat[:, 0] = np.minimum(zq / Z_FAR, 1.0)
    feat[:, 1:4] = np.asarray(normal, np.float64).reshape(P, 3)[q]
    feat[:, 4] = (fmix32(np.asarray(ids).reshape(P)[q]) >> np.uint32(8)).astype(np.float64) * 2.0 ** -24
    feat[:, 5:8] = np.asarray(rgb, np.float64).reshape(P, 3)[q]
    feat[:, 8] = D[q].astype(np.float64) * DISP_SCALE
    if refl is not None:
        feat[:, 9] = np.asarray(refl, np.float32).reshape(P)[q].astype(np.float64)
    feat[hole] = 0.0
    return feat, hole, feat[:, 5:8].copy(), source


def labels(hole, warped, full, threshold=1e-2):
    err = np.abs(np.asarray(warped, np.float64) - np.asarray(full, np.float64)).max(axis=-1)
    return (np.asarray(hole, bool) | (err > threshold)).astype(np.float64)


# ------------------------------------------------------------------ network
def unpack(params):
    p = np.asarray(params, np.float64).reshape(-1)
    out, k = [], 0
    for ci, co in LAYERS:
        w = p[k:k + co * ci * 9].reshape(co, ci, 3, 3)
        k += co * ci * 9
        b = p[k:k + co]
        k += co
        out.append((w, b))
    assert k == p.size
    return out


def _bf16(t):
    import torch
    return t.to(torch.bfloat16).to(torch.float64)


def forward(params, feat, W, H, bf16=True):
    """Retrace probability (H, W) of features (P, >= IN_CH), float64."""
    import torch
    import torch.nn.functional as F
    x = torch.tensor(np.asarray(feat, np.float64)[:, :IN_CH].reshape(H, W, IN_CH)).permute(2, 0, 1)[None]
    if bf16:
        x = _bf16(x)
    layers = unpack(params)
    for li, (w, b) in enumerate(layers):
        wt = torch.tensor(w)
        if bf16:
            wt = _bf16(wt)
        x = F.conv2d(x, wt, torch.tensor(b), padding=1)
        if li < 3:
            x = torch.relu(x)
            if bf16:
                x = _bf16(x)
    return torch.sigmoid(x)[0, 0].numpy()


E4M3_MAX = 448.0


def e4m3(x):
    """Round to the nearest OCP FP8 E4M3 value (ties to even), saturating at
    +-448, in float64. Spacing 2^(e-3) in the binade [2^e, 2^(e+1)) for
    e >= -6, and 2^-9 below 2^-6 (subnormals)."""
    x = np.asarray(x, np.float64)
    a = np.abs(x)
    _, k = np.frexp(np.where(a > 0, a, 1.0))          # a = m 2^k, m in [0.5, 1)
    e = np.maximum(k.astype(np.float64) - 1.0, -6.0)  # floor(log2 a), at least -6
    q = np.exp2(e - 3.0)
    r = np.minimum(np.round(a / q) * q, E4M3_MAX)      # np.round: half to even
    return np.copysign(r, x)


def pow2_scale(amax):
    """Largest power of two s with amax * s <= 448 (1 when amax is 0): 2^(k-1)
    for 448 / amax = m 2^k, m in [0.5, 1)."""
    amax = np.asarray(amax, np.float64)
    ratio = np.where(amax > 0, E4M3_MAX / np.where(amax > 0, amax, 1.0), 2.0)
    _, k = np.frexp(ratio)
    return np.where(amax > 0, np.ldexp(1.0, k - 1), 1.0)


def weight_scales_fp8(params):
    """Per-output-channel scales of layers 2-4: pow2_scale of the largest
    |weight| of the channel, taken over the float32 parameters."""
    layers = unpack(np.asarray(params, np.float32).astype(np.float64))
    return [pow2_scale(np.abs(w).reshape(w.shape[0], -1).max(axis=1)) for w, _ in layers[1:]]


def forward_fp8(params, feat, W, H, act_scales):
    """Retrace probability (H, W) of the FP8 network, float64 arithmetic.
    act_scales: scales of the three hidden activations (layer 1-3 outputs)."""
    import torch
    import torch.nn.functional as F
    x = torch.tensor(np.asarray(feat, np.float64)[:, :IN_CH].reshape(H, W, IN_CH)).permute(2, 0, 1)[None]
    x = _bf16(x)
    layers = unpack(params)
    wsc = weight_scales_fp8(params)
    w0, b0 = layers[0]
    z = F.conv2d(x, _bf16(torch.tensor(w0)), torch.tensor(b0), padding=1)
    q = torch.tensor(e4m3(torch.relu(z).numpy() * act_scales[0]))     # stored activation
    for li in (1, 2, 3):
        w, b = layers[li]
        s_w = wsc[li - 1]
        wq = torch.tensor(e4m3(np.asarray(w, np.float32).astype(np.float64) * s_w[:, None, None, None]))
        acc = F.conv2d(q, wq, None, padding=1)
        inv = torch.tensor(1.0 / (act_scales[li - 1] * s_w))[None, :, None, None]
        z = acc * inv + torch.tensor(b)[None, :, None, None]
        if li < 3:
            q = torch.tensor(e4m3(torch.relu(z).numpy() * act_scales[li]))
    return torch.sigmoid(z)[0, 0].numpy()


def loss_and_grads(params, feat, label, W, H):
    """Mean BCE of the float64 network and its gradient (parameter layout)."""
    import torch
    import torch.nn.functional as F
    p = torch.tensor(np.asarray(params, np.float64).reshape(-1), requires_grad=True)
    x = torch.tensor(np.asarray(feat, np.float64)[:, :IN_CH].reshape(H, W, IN_CH)).permute(2, 0, 1)[None]
    k = 0
    for li, (ci, co) in enumerate(LAYERS):
        w = p[k:k + co * ci * 9].reshape(co, ci, 3, 3)
        k += co * ci * 9
        b = p[k:k + co]
        k += co
        x = F.conv2d(x, w, b, padding=1)
        if li < 3:
            x = torch.relu(x)
    q = torch.sigmoid(x)[0, 0].reshape(-1)
    y = torch.tensor(np.asarray(label, np.float64).reshape(-1))
    loss = -(y * torch.log(q) + (1 - y) * torch.log(1 - q)).mean()
    loss.backward()
    return float(loss.item()), p.grad.numpy().copy()


def grads_emulated(params, feat, label, W, H, bf16=True):
    """Mean-BCE gradient by an explicit backward pass (float64) that rounds
    to BF16 where the tensor-core kernels do: inputs, weights and hidden
    activations of the forward pass, the data gradients after the ReLU mask,
    and the (p - y) map fed to the layer-4 data gradient; the layer-4 weight
    gradient uses p - y unrounded. With bf16=False it is the plain gradient."""
    import torch
    import torch.nn.functional as F
    from torch.nn import grad as G
    rb = _bf16 if bf16 else (lambda t: t)
    P = W * H
    layers = [(torch.tensor(w), torch.tensor(b)) for w, b in unpack(params)]
    a = [rb(torch.tensor(np.asarray(feat, np.float64)[:, :IN_CH].reshape(H, W, IN_CH)).permute(2, 0, 1)[None])]
    for li in range(3):
        w, b = layers[li]
        a.append(rb(torch.relu(F.conv2d(a[-1], rb(w), b, padding=1))))
    w4, b4 = layers[3]
    q = torch.sigmoid(F.conv2d(a[3], rb(w4), b4, padding=1))
    y = torch.tensor(np.asarray(label, np.float64).reshape(1, 1, H, W))
    g = q - y
    grads = []
    dz = g
    dz_in = rb(g)
    for li in (3, 2, 1, 0):
        w, b = layers[li]
        grads.append((G.conv2d_weight(a[li], w.shape, dz, padding=1) / P, dz.sum(dim=(0, 2, 3)) / P))
        if li > 0:
            da = G.conv2d_input(a[li].shape, rb(w), dz_in, padding=1)
            dz = rb(da * (a[li] > 0))
            dz_in = dz
    out = []
    for dw, db in reversed(grads):
        out += [dw.reshape(-1), db.reshape(-1)]
    return torch.cat(out).numpy()
