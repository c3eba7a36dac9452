"""Train and evaluate the retrace network of the learned right-eye reprojection.

Training data: config-1-style scenes (8 random spheres on a ground plane,
one light, reflection depth 3), seeds 1000..1199, traced in full at 960x540
per eye by the GPU tracer; each right-eye pixel is labelled 1 where it is a
disocclusion hole or its warped colour differs from the full trace by more
than 1e-2 in some channel. The network (3x3 convolutions 9 -> 32 -> 32 -> 32
-> 1) is trained with Adam on the mean binary cross-entropy by the library's
own tensor-core kernels (rt_net_train_step). Held-out seeds 2000..2009 at
1920x1080 choose the retrace threshold: the largest one whose right-eye PSNR
against the full trace is >= 40 dB on every held-out scene.

    python -m paper_1702_01530_gb300.train_reproj --out weights.bin

Weights file: magic b"RTNET1\\0\\0", uint32 parameter count, float32
parameters, float32 threshold, uint32 CRC-32 of everything before it.
"""
from __future__ import annotations

import argparse
import binascii
import json
import os
import struct
import time

import numpy as np

from . import capi, scenegen as sg

MAGIC = b"RTNET1\0\0"
DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                               "reproj_net.bin")
THRESHOLDS = (0.9, 0.7, 0.5, 0.35, 0.25, 0.15, 0.1, 0.06, 0.03, 0.015, 0.0075)


def save_weights(path: str, params: np.ndarray, threshold: float):
    p = np.ascontiguousarray(params, np.float32)
    body = MAGIC + struct.pack("<I", p.size) + p.tobytes() + struct.pack("<f", threshold)
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "wb") as f:
        f.write(body + struct.pack("<I", binascii.crc32(body) & 0xFFFFFFFF))


def load_weights(path: str = DEFAULT_WEIGHTS):
    data = open(path, "rb").read()
    if data[:8] != MAGIC:
        raise ValueError(f"{path}: not a retrace-network weights file")
    body, crc = data[:-4], struct.unpack("<I", data[-4:])[0]
    if binascii.crc32(body) & 0xFFFFFFFF != crc:
        raise ValueError(f"{path}: CRC mismatch")
    (n,) = struct.unpack("<I", body[8:12])
    params = np.frombuffer(body[12:12 + 4 * n], np.float32).copy()
    (thr,) = struct.unpack("<f", body[12 + 4 * n:16 + 4 * n])
    if n != capi.RT_NET_PARAMS:
        raise ValueError(f"{path}: {n} parameters, expected {capi.RT_NET_PARAMS}")
    return params, float(thr)


def make_dataset(seeds, W, H):
    """Features (BF16, P x 16) and labels (P) of each seed, kept on the GPU."""
    import torch
    data = []
    P = W * H
    L = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    R = torch.empty_like(L)
    for seed in seeds:
        s = sg.config_small(seed, W=W, H=H)
        g = capi.GpuScene(s)
        f16 = torch.empty((P, 16), dtype=torch.bfloat16, device="cuda")
        lab = torch.empty(P, dtype=torch.float32, device="cuda")
        capi.rt_reproj_training_pair(g.handle, s.camera, s.eye_sep, s.convergence, W, H,
                                     s.max_depth, L, R, f16, lab, 1e-2)
        capi.rt_sync_status(g.handle)
        g.close()
        data.append((f16, lab))
    return data


def train(data, W, H, epochs=8, lr=1e-3, seed=0, log=print):
    net = capi.Net(sg.net_params_he(seed))
    order = np.random.default_rng(seed)
    history = []
    for ep in range(epochs):
        idx = order.permutation(len(data))
        losses = []
        for k, i in enumerate(idx):
            f16, lab = data[i]
            want = k % 25 == 0 or k == len(idx) - 1
            loss = capi.rt_net_train_step(net.handle, f16, lab, W, H, lr, want_loss=want)
            if want:
                losses.append(loss)
        capi.rt_net_status(net.handle)
        history.append(float(np.mean(losses)))
        log(f"epoch {ep}: mean sampled loss {history[-1]:.4f}")
    return net, history


def fp8_calibrate(net_handle, seeds=(2000, 2001, 2002), W=1920, H=1080):
    """Switch a network to FP8 inference with activation scales chosen by the
    library (rt_net_calibrate_fp8) from the reprojection features of held-out
    small scenes; returns the scales."""
    import torch
    P = W * H
    L = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    R = torch.empty_like(L)
    lab = torch.empty(P, dtype=torch.float32, device="cuda")
    feats = []
    for seed in seeds:
        s = sg.config_small(seed, W=W, H=H)
        g = capi.GpuScene(s)
        f16 = torch.empty((P, 16), dtype=torch.bfloat16, device="cuda")
        capi.rt_reproj_training_pair(g.handle, s.camera, s.eye_sep, s.convergence, W, H,
                                     s.max_depth, L, R, f16, lab, 1e-2)
        capi.rt_sync_status(g.handle)
        g.close()
        feats.append(f16)
    _, scales = capi.rt_net_calibrate_fp8(net_handle, feats, W, H)
    return scales


def psnr(a, b) -> float:
    import torch
    mse = torch.mean((a - b) ** 2).item()
    return 10.0 * np.log10(1.0 / max(mse, 1e-20))


def _time_ms(fn, reps=20, warm=5):
    import torch
    for _ in range(warm):
        fn()
    st = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def evaluate(net_handle, seeds, W, H, thresholds=THRESHOLDS, time_it=True, make_scene=None):
    """Right-eye PSNR, retraced fraction and time of full vs reprojected pairs
    for each threshold (net_handle None: holes only)."""
    import torch
    make_scene = make_scene or (lambda seed: sg.config_small(seed, W=W, H=H))
    P = W * H
    rows = []
    for seed in seeds:
        s = make_scene(seed)
        g = capi.GpuScene(s)
        img = torch.empty((2, H, W, 3), dtype=torch.float32, device="cuda")
        L = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
        R = torch.empty_like(L)
        n = torch.zeros(1, dtype=torch.int32, device="cuda")
        st = torch.cuda.current_stream()

        def full():
            capi.rt_render_stereo(g.handle, s.camera, s.eye_sep, s.convergence, W, H, s.max_depth,
                                  img[0], img[1], st)

        full()
        capi.rt_sync_status(g.handle)
        t_full = _time_ms(full) if time_it else None
        for thr in (thresholds if net_handle is not None else (1.0,)):
            def rep():
                capi.rt_render_stereo_reproj(g.handle, s.camera, s.eye_sep, s.convergence, W, H,
                                             s.max_depth, net_handle, thr, L, R, n, st)
            rep()
            capi.rt_sync_status(g.handle)
            row = {"seed": seed, "threshold": thr if net_handle is not None else None,
                   "psnr": psnr(R, img[1]), "retraced": int(n.item()) / P,
                   "left_exact": bool(torch.equal(L, img[0]))}
            if time_it:
                row["ms_full"] = t_full
                row["ms_reproj"] = _time_ms(rep)
                row["speedup"] = t_full / row["ms_reproj"]
            rows.append(row)
        g.close()
    return rows


def choose_threshold(rows, target_db=40.0):
    """The largest threshold whose PSNR reaches target_db on every scene."""
    by = {}
    for r in rows:
        by.setdefault(r["threshold"], []).append(r)
    ok = [t for t, rs in by.items() if min(r["psnr"] for r in rs) >= target_db]
    return max(ok) if ok else min(by)


def summarise(rows, thr):
    rs = [r for r in rows if r["threshold"] == thr]
    out = {"threshold": thr, "psnr_min": min(r["psnr"] for r in rs),
           "psnr_mean": float(np.mean([r["psnr"] for r in rs])),
           "retraced_mean": float(np.mean([r["retraced"] for r in rs]))}
    if "speedup" in rs[0]:
        out.update(ms_full=float(np.mean([r["ms_full"] for r in rs])),
                   ms_reproj=float(np.mean([r["ms_reproj"] for r in rs])),
                   speedup=float(np.mean([r["speedup"] for r in rs])))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-seeds", type=int, default=200)
    ap.add_argument("--eval-seeds", type=int, default=10)
    ap.add_argument("--W", type=int, default=960)
    ap.add_argument("--H", type=int, default=540)
    ap.add_argument("--eval-W", type=int, default=1920)
    ap.add_argument("--eval-H", type=int, default=1080)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--report", default=None, help="write the evaluation as JSON here")
    a = ap.parse_args()
    from . import build
    build.build()
    t0 = time.time()
    data = make_dataset(range(1000, 1000 + a.train_seeds), a.W, a.H)
    pos = float(np.mean([d[1].mean().item() for d in data]))
    print(f"dataset: {len(data)} scenes at {a.W}x{a.H}, positive fraction {pos:.4f}, "
          f"{time.time() - t0:.1f} s")
    t1 = time.time()
    net, hist = train(data, a.W, a.H, epochs=a.epochs, lr=a.lr)
    print(f"trained in {time.time() - t1:.1f} s")
    del data
    eval_seeds = range(2000, 2000 + a.eval_seeds)
    rows = evaluate(net.handle, eval_seeds, a.eval_W, a.eval_H)
    thr = choose_threshold(rows)
    base = evaluate(None, eval_seeds, a.eval_W, a.eval_H)
    rep = {"train": {"scenes": a.train_seeds, "W": a.W, "H": a.H, "epochs": a.epochs,
                     "lr": a.lr, "positive_fraction": pos, "loss_per_epoch": hist},
           "chosen": summarise(rows, thr), "holes_only": summarise(base, None),
           "per_threshold": [summarise(rows, t) for t in THRESHOLDS]}
    save_weights(a.out, net.params(), thr)
    print(json.dumps(rep, indent=1))
    if a.report:
        json.dump({"report": rep, "rows": rows, "holes_only_rows": base}, open(a.report, "w"),
                  indent=1)
    net.close()


if __name__ == "__main__":
    main()
