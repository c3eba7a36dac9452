"""Row-band split of a stereo pair over several GPUs (one process per GPU).

Paper Sec. 3, Figure 1: the image is divided into N parts and each
processor renders its part. Here rank r of N renders rows
``row_bands(H, N)[r]`` of both eyes with ``rt_render_stereo_rows`` over its
own copy of the scene; the bands need no exchange while they are traced
(every pixel is independent), and ``gather_bands`` collects the finished
bands into whole images on rank 0 -- the only collective, after the trace.
Bands are horizontal because off-axis stereo has horizontal disparity only:
a band holds everything the learned reprojection of its rows needs.
"""
from __future__ import annotations


def row_bands(H: int, n: int) -> list[tuple[int, int]]:
    """(row0, n_rows) of each of n bands covering rows 0..H-1 in order; the
    first H % n bands get one row more. Ranks beyond H get empty bands."""
    if H < 0 or n < 1:
        raise ValueError("need H >= 0 and n >= 1")
    base, extra = divmod(H, n)
    out, r0 = [], 0
    for r in range(n):
        k = base + (1 if r < extra else 0)
        out.append((r0, k))
        r0 += k
    return out


def gather_bands(band_L, band_R, H: int, rank: int, world: int):
    """All-gather each rank's band (n_rows x W x 3 tensors of both eyes) and
    stitch them in row order: returns the whole (H, W, 3) images on rank 0,
    None on the other ranks. Bands are padded to the tallest band for the
    collective (torch.distributed all_gather wants equal shapes)."""
    import torch
    import torch.distributed as dist
    bands = row_bands(H, world)
    tall = max(k for _, k in bands)
    W = band_L.shape[1]
    pair = torch.zeros((2, tall, W, 3), dtype=band_L.dtype, device=band_L.device)
    k = bands[rank][1]
    pair[0, :k] = band_L[:k]
    pair[1, :k] = band_R[:k]
    parts = [torch.empty_like(pair) for _ in range(world)]
    dist.all_gather(parts, pair)
    if rank != 0:
        return None
    full = torch.empty((2, H, W, 3), dtype=band_L.dtype, device=band_L.device)
    for (r0, kk), p in zip(bands, parts):
        full[:, r0:r0 + kk] = p[:, :kk]
    return full[0], full[1]
