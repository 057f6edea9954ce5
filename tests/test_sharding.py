"""Multi-GPU host logic of bench.py on CPU: two gloo ranks own disjoint
channel ranges that together equal a single-process batch, and the job
throughput uses the slowest rank's time.  No data-path collective exists."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, n, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_2305_13925_gb300 import channels as C
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        a, b = bench.shard_range(rank, n)
        Hst, xi = C.generate_batch_device_layout("single_256x16", n, 5, first=a, workers=1)
        t_ms = 10.0 + 5.0 * rank                      # pretend rank 1 is slower
        t_max = bench.reduce_max(t_ms, dist)
        out[rank] = (a, b, Hst, xi, t_max, bench.job_throughput(n, world, 3, t_max))
    finally:
        dist.destroy_process_group()


def test_two_rank_weak_scaling_shards():
    n, world = 3, 2
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, n, out), nprocs=world, join=True,
                       start_method="spawn")
    from paper_2305_13925_gb300 import channels as C
    full, xi_full = C.generate_batch_device_layout("single_256x16", n * world, 5, workers=1)
    got = [out[r] for r in range(world)]
    assert [(g[0], g[1]) for g in got] == [(0, 3), (3, 6)]
    assert np.array_equal(np.concatenate([g[2] for g in got]), full)
    assert np.array_equal(np.concatenate([g[3] for g in got]), xi_full)
    for g in got:
        assert g[4] == 15.0                            # max over ranks
        assert abs(g[5] - n * world * 3 / 0.015) < 1e-6
