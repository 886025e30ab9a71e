"""Multi-rank (replica) logic of bench.py on CPU: two gloo ranks on
127.0.0.1 check that the replicas' realization seeds never collide, that the
job time is the slowest rank's, and that the whole-job throughput counts
every rank's realizations.  No GPU and no CUDA call."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        batch, steps, warm = 8, 5, 3
        mine = [s for k in range(warm + steps) for s in bench.replica_seeds(100, batch, k, rank)]
        everyone = [None] * world
        dist.all_gather_object(everyone, mine)
        ms = 1000.0 + 250.0 * rank            # the ranks' own step times
        ms_max = bench.max_over_ranks(ms, dist, "cpu")
        value = bench.job_throughput(batch, steps, world, ms_max)
        out.put((rank, everyone, ms_max, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, everyone, ms_max, value in res:
        flat = [s for seeds in everyone for s in seeds]
        assert len(flat) == len(set(flat))            # no seed reused anywhere
        assert ms_max == 1250.0                       # slowest rank's time on every rank
        assert value == pytest.approx(8 * 5 * 2 / 1.25)


def test_replica_seeds_disjoint_single_process():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    seen = set()
    for rank in range(8):
        for k in range(99):
            s = bench.replica_seeds(7, 64, k, rank)
            assert not seen.intersection(s)
            seen.update(s)
