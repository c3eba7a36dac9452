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
