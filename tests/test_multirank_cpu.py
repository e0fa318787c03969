"""The N-rank host logic on CPU ranks (gloo, world size 2): the timing
barrier and the max over ranks that bench.py applies to every rank's time,
and the row-sharded exchange of pass 1 -- each rank's aggregates of its
rows (the paper's per-worker partial sums, Sec. III-A) summed over ranks
equal the aggregates of all rows.  Failures are made on the host: a rank
that leaves between steps ends the survivor's next collective with an error
(a short process-group timeout, never a hang), and a shard that goes missing
from the merge shows in the counts, which must add up to N."""
import datetime
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


def _rank_that_may_leave(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    import bench
    bench.barrier(world)
    out[f"step0_{rank}"] = bench.max_over_ranks(1.0 + rank, world, device="cpu")
    if rank == 1:
        out["left"] = True
        os._exit(0)  # leaves between steps, with nothing in flight
    try:
        bench.max_over_ranks(2.0, world, device="cpu")  # the next step's collective
        out["detected"] = "none"
    except Exception as e:  # noqa: BLE001 -- any error ends the step; a hang would not
        out["detected"] = type(e).__name__
    os._exit(0)


def test_a_rank_that_leaves_is_detected_by_the_next_collective():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_that_may_leave, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank hung instead of failing its collective"
    assert out["step0_0"] == out["step0_1"] == 2.0  # the step before the failure completed
    assert out["left"] is True
    assert out["detected"] != "none"


def test_a_missing_shard_shows_in_the_counts():
    # aggregates are sums over rows: merged over every shard the counts add up
    # to N; with a shard lost they do not (and S would come from the wrong
    # clusters), which a caller merging shards can check before scoring
    import oracle
    from paper_2303_14102_gb300 import synth
    w = synth.workload_small(N=3000, D=5, K=4)
    X, lab = w.X.double().numpy(), w.labels.numpy()
    shards = [oracle.aggregate(X[r::3], lab[r::3], w.K) for r in range(3)]
    full = sum(int(c.sum()) for c, _, _ in shards)
    lost = sum(int(c.sum()) for c, _, _ in shards[:2])
    assert full == X.shape[0]
    assert lost != X.shape[0]
