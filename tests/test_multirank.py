"""Host logic of the N > 1 benchmark path on CPU: world_size-2 gloo ranks.
The path shards by replica (templates and segments are independent, so each
rank filters its own seeded replica and no data moves between ranks); the
only exchange is the max-over-ranks of the timed region."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads
    ms = [40.0, 55.0][rank]                       # rank 1 is the slowest
    tmax = bench.max_over_ranks(ms, dist, "cpu")
    rate = bench.whole_job_rate(world, 1024 * 10, tmax)
    wl = workloads.scale(seed=rank)               # each rank's own replica
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, tmax, rate, float(wl.m1[0]), int(wl.segments[0].seed)))


@pytest.mark.timeout(120)
def test_two_gloo_ranks_share_the_slowest_time():
    pytest.importorskip("torch")
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=100) for _ in ps)
    for p in ps:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [55.0, 55.0]                  # max over ranks on every rank
    assert res[0][2] == res[1][2] == pytest.approx(2 * 1024 * 10 / 0.055)
    assert res[0][4] != res[1][4]                               # distinct seeded replicas


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 3
    assert bench.run_reference(A()) == 0
