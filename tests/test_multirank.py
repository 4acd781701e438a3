"""The N > 1 path of the benchmark on CPU: two gloo ranks each take their own
seeded batch (weak scaling, no exchange on the data path) and agree on the
slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    wl = bench.rank_workload(rank, 8, 10)
    t = bench.max_over_ranks(1.0 + rank, dist)
    sizes = [int(i.nz) for i in wl.instances]
    gathered = [None] * world
    dist.all_gather_object(gathered, sizes)
    out.put((rank, t, gathered))
    dist.destroy_process_group()


def test_two_ranks_shard_and_agree_on_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, gathered in res:
        assert t == 2.0                       # the slower rank's time
        assert gathered[0] != gathered[1]     # each rank has its own batch
    assert res[0][2] == res[1][2]
