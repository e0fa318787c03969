"""The N-rank host logic on CPU ranks (gloo, world size 2): the timing
barrier and the max over ranks that bench.py applies to every rank's time,
and the row-sharded exchange of pass 1 -- each rank's aggregates of its
rows (the paper's per-worker partial sums, Sec. III-A) summed over ranks
equal the aggregates of all rows."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        from paper_2303_14102_gb300 import synth
        bench.barrier(world)
        m = bench.max_over_ranks(1.5 + rank, world, device="cpu")
        w = synth.workload_small(N=2000, D=6, K=4)
        X, lab = w.X.double().numpy(), w.labels.numpy()
        c, s1, s2 = oracle.aggregate(X[rank::world], lab[rank::world], w.K)
        t = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)) for a in (c, s1, s2)]
        for a in t:
            dist.all_reduce(a)
        out[rank] = (m, [a.numpy() for a in t])
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks_time_max_and_sharded_aggregates():
    import oracle
    from paper_2303_14102_gb300 import synth
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w = synth.workload_small(N=2000, D=6, K=4)
    c, s1, s2 = oracle.aggregate(w.X.double().numpy(), w.labels.numpy(), w.K)
    for r in range(world):
        m, (rc, rs1, rs2) = out[r]
        assert m == 1.5 + (world - 1)  # every rank reports the slowest rank's time
        np.testing.assert_array_equal(rc, c)
        np.testing.assert_allclose(rs1, s1, rtol=1e-12, atol=1e-9)
        np.testing.assert_allclose(rs2, s2, rtol=1e-12, atol=1e-9)
