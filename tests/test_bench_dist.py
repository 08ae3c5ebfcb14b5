"""The bench's N > 1 path on the CPU: two gloo ranks, each stepping its own replica, aggregate
to (sum of node updates) / (slowest rank's time)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, l = bench.dist_setup()
        assert (w, r, l) == (world, rank, rank)
        units = 1000.0 * (rank + 1)
        secs = 0.5 + rank
        q.put((rank, bench.aggregate(units, secs, world)))
    finally:
        dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert out[r] == pytest.approx((3000.0, 1.5))


def test_aggregate_single_rank():
    import bench
    assert bench.aggregate(10.0, 2.0, 1) == (10.0, 2.0)


def test_kernel_hash_ignores_comments_not_code():
    """The hash that ties the committed ncu counts to the kernel source changes with the code and
    not with comments or layout (a `//` inside a string literal is code)."""
    import bench
    base = 'int x; // a comment\n  /* block\n comment */ asm("add %0; // in string");\n'
    same = 'int x;\nasm("add %0; // in string");'
    assert bench._code_only(base) == bench._code_only(same)
    assert bench._code_only(base) != bench._code_only(same.replace("x", "y"))
    assert bench._code_only(base) != bench._code_only(same.replace("in string", "in strung"))
