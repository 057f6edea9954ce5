"""Multi-GPU logic on CPU with gloo ranks.  bench.py's sharding: two ranks
own disjoint channel ranges that together equal a single-process batch, and
the job throughput uses the slowest rank's time; the product path has no
data-path collective.  The within-instance split by subarray (partial Grams
summed by one all-reduce) is checked on the oracle."""
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


def _subarray_rank(rank, world, port, out):
    import sys
    import torch
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle import oracle as O
    from paper_2305_13925_gb300 import channels as C
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        inst = C.generate_instance(C.PRESETS["single_256x16"], 7, 0)
        H, xi = inst.H, inst.xi
        rows = H.shape[0] // world
        Hr = H[rank * rows:(rank + 1) * rows]          # this rank's subarrays
        G = O.gram(Hr, 0.0)                              # partial Gram H_r^H H_r
        g = torch.from_numpy(np.stack([G.real, G.imag]))
        dist.all_reduce(g, op=dist.ReduceOp.SUM)         # the one exchange of the path
        A = g[0].numpy() + 1j * g[1].numpy() + xi * np.eye(H.shape[1])
        X, _, _, st = O.pcg(A, None, "standard", max_iter=8)   # replicated on every rank
        Wr = O.matmul(Hr, X)                             # local rows of W, no exchange
        w2 = torch.tensor([float(np.sum(np.abs(Wr) ** 2))], dtype=torch.float64)
        dist.all_reduce(w2, op=dist.ReduceOp.SUM)        # scalar for the power factor
        out[rank] = (Wr, float(np.sqrt(1.0 / w2.item())), st)
    finally:
        dist.destroy_process_group()


def test_two_rank_subarray_decomposition():
    """The within-instance split across ranks (Sec. II: one processing unit per
    subarray): rows of H partitioned by subarray, partial Grams summed by one
    all-reduce, the iteration replicated on A, each rank forming its rows of
    W = H X; one scalar all-reduce gives the power factor.  The stacked result
    equals the single-process precoder.  Checked on the oracle with gloo
    ranks; every GPU machine has one GPU, so the product path runs replicas only."""
    from oracle import oracle as O
    from paper_2305_13925_gb300 import channels as C
    O.lib()                                              # build once, before the ranks load it
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_subarray_rank, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    inst = C.generate_instance(C.PRESETS["single_256x16"], 7, 0)
    ref = O.precode(inst.H, inst.xi, "standard", max_iter=8)
    W = np.concatenate([out[r][0] for r in range(world)])
    assert all(out[r][2] == 0 for r in range(world))
    assert np.linalg.norm(W - ref["W"]) <= 1e-12 * np.linalg.norm(ref["W"])
    for r in range(world):
        assert abs(out[r][1] - ref["beta"]) <= 1e-12 * ref["beta"]
