"""The multi-GPU bench path on CPU: N ranks run independent replicas and
combine only their times (max over ranks), over a world_size-2 gloo group."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
        val = bench.replica_throughput(1000, world, 2, ms)
        q.put((rank, ms, val, bench.dist_info()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, val, info in out:
        assert ms == 20.0  # the slower rank's time
        assert val == pytest.approx(2 * 1000 * 2 / 0.020)
        assert info[0] == rank and info[1] == 2


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.replica_throughput(10, 1, 1, 1000.0) == 10.0


@pytest.mark.parametrize("kind,dtype", [("list", "u64"), ("tree", "u64"), ("scan", "u32"), ("scan", "u64")])
def test_workload_cpu_baseline_is_a_bounded_oracle_timing(kind, dtype):
    # The list, tree and scan lines time their oracle on one host thread over
    # a bounded sample, repeating on copies of one input up to a cap.
    import bench

    cb = bench.cpu_oracle_workload(kind, 0.5, 3, 4096, dtype, min_seconds=0.05, max_reps=3)
    assert set(cb) == {"value", "unit", "cores", "kind", "sample"}
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] > 0
    assert cb["unit"] == ("elems/s" if kind == "scan" else "nodes/s")
    reps = int(cb["sample"].split(" runs on copies")[0].rsplit(", ", 1)[1])
    assert 1 <= reps <= 3
