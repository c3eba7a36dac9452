"""The multi-GPU host logic of bench.py as world-size-2 gloo ranks on CPU.

The path shards into independent replicas (every pixel and eye is
independent; the paper's Figure 1 split), so the only cross-rank steps are a
barrier around the timed region and the maximum of the per-rank step times;
rank 0 prints the line. No GPU is needed for these steps.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_setup(None)
        dist.barrier()
        # rank-dependent step times: the job's time is the slowest rank's
        ms, e2e = bench.max_over_ranks([1.0 + rank, 2.5 - rank], w)
        mrays, pairs = bench.job_rates(6_000_000, w, ms)
        queue.put((r, w, local, ms, e2e, mrays, pairs))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_agree_on_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, queue)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(queue.get(timeout=90) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, (r, w, local, ms, e2e, mrays, pairs) in enumerate(out):
        assert (r, w, local) == (rank, 2, rank)
        assert ms == 2.0 and e2e == 2.5          # max over ranks of (1, 2) and (2.5, 1.5)
        assert mrays == pytest.approx(2 * 6_000_000 / 2e-3 / 1e6)   # both replicas' rays
        assert pairs == pytest.approx(2 / 2e-3)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 3.0], 1) == [1.5, 3.0]
    assert bench.job_rates(1_000_000, 1, 1.0) == pytest.approx((1000.0, 1000.0))


# ------------------------------------------------------------ row bands
def test_row_bands_partition():
    from paper_1702_01530_gb300.bands import row_bands
    assert row_bands(10, 3) == [(0, 4), (4, 3), (7, 3)]
    assert row_bands(1080, 8) == [(135 * r, 135) for r in range(8)]
    assert row_bands(2, 4) == [(0, 1), (1, 1), (2, 0), (2, 0)]
    for H in (1, 7, 61, 1080):
        for n in (1, 2, 3, 5, 8):
            b = row_bands(H, n)
            assert sum(k for _, k in b) == H and b[0][0] == 0
            assert all(b[i][0] + b[i][1] == b[i + 1][0] for i in range(n - 1))
            assert max(k for _, k in b) - min(k for _, k in b) <= 1


def _band_rank(rank, world, port, H, W, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_1702_01530_gb300.bands import gather_bands, row_bands
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank "renders" its band of a known image: value = row * 1000 + col (+0.5 right eye)
        r0, k = row_bands(H, world)[rank]
        rows = torch.arange(r0, r0 + k, dtype=torch.float32)[:, None, None]
        cols = torch.arange(W, dtype=torch.float32)[None, :, None]
        band_L = (rows * 1000 + cols).expand(k, W, 3).contiguous()
        band_R = band_L + 0.5
        out = gather_bands(band_L, band_R, H, rank, world)
        if rank == 0:
            L, R = out
            queue.put((rank, L.numpy().copy(), R.numpy().copy()))
        else:
            queue.put((rank, out, None))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_gather_uneven_bands_in_row_order():
    import numpy as np
    world, H, W = 2, 7, 5
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_band_rank, args=(r, world, port, H, W, queue)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict((r, (a, b)) for r, a, b in (queue.get(timeout=90) for _ in range(world)))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    want = (np.arange(H)[:, None] * 1000 + np.arange(W)[None, :]).astype(np.float32)
    L, R = out[0]
    assert np.array_equal(L, np.repeat(want[:, :, None], 3, axis=2))
    assert np.array_equal(R, L + 0.5)
    assert out[1] == (None, None)
