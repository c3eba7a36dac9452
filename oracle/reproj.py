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
  (fmix32(id) >> 8) 2^-24 (MurmurHash3 finaliser), left RGB, D/16; zeros on a
  hole. Labels: hole or max_c |warped - full| > threshold.
* network: 3x3 convolutions 9 -> 32 -> 32 -> 32 -> 1 with zero padding 1,
  ReLU, sigmoid; mean binary cross-entropy; gradients by autograd in float64.
  `forward(..., bf16=True)` rounds inputs, weights and hidden activations to
  BF16 where the tensor-core kernels do, so the two can be compared closely.
"""
from __future__ import annotations

import numpy as np

Z_FAR = 100.0
DISP_SCALE = 1.0 / 16.0
LAYERS = ((9, 32), (32, 32), (32, 32), (32, 1))


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


def warp(depth, normal, ids, rgb, W, H, f_px, eye_sep, convergence):
    """Returns features (P, 9) float64, hole (P,) bool, warped RGB (P, 3),
    source index (P,) int64 (-1 on a hole)."""
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
    feat = np.zeros((P, 9), np.float64)
    zq = z[q].astype(np.float64)
    with np.errstate(invalid="ignore"):
        feat[:, 0] = np.minimum(zq / Z_FAR, 1.0)
    feat[:, 1:4] = np.asarray(normal, np.float64).reshape(P, 3)[q]
    feat[:, 4] = (fmix32(np.asarray(ids).reshape(P)[q]) >> np.uint32(8)).astype(np.float64) * 2.0 ** -24
    feat[:, 5:8] = np.asarray(rgb, np.float64).reshape(P, 3)[q]
    feat[:, 8] = D[q].astype(np.float64) * DISP_SCALE
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
    """Retrace probability (H, W) of features (P, >=9), float64."""
    import torch
    import torch.nn.functional as F
    x = torch.tensor(np.asarray(feat, np.float64)[:, :9].reshape(H, W, 9)).permute(2, 0, 1)[None]
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


def loss_and_grads(params, feat, label, W, H):
    """Mean BCE of the float64 network and its gradient (parameter layout)."""
    import torch
    import torch.nn.functional as F
    p = torch.tensor(np.asarray(params, np.float64).reshape(-1), requires_grad=True)
    x = torch.tensor(np.asarray(feat, np.float64)[:, :9].reshape(H, W, 9)).permute(2, 0, 1)[None]
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
    a = [rb(torch.tensor(np.asarray(feat, np.float64)[:, :9].reshape(H, W, 9)).permute(2, 0, 1)[None])]
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
