"""The multi-GPU host logic (one replica per rank, MAX of the timings, units
summed over ranks) on CPU with gloo, world size 2."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1002_3094_gb300 import replicas as RP  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = RP.rank_env()
        inst = RP.replica_instance(r)
        # each rank's timing and units differ; the job takes the slowest time
        # and the units of all ranks
        secs = 1.0 + r
        units = 100.0 * (r + 1)
        t = RP.max_over_ranks(secs, dist, "cpu")
        rate = RP.aggregate_rate(units, t, dist, "cpu")
        insts = [None] * world
        dist.all_gather_object(insts, inst)
        q.put((r, w, lr, t, rate, insts))
    finally:
        dist.destroy_process_group()


def test_replicas_gloo_world_2():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, lr, t, rate, insts in out:
        assert w == world and lr == r
        assert t == 2.0                         # the slower rank's time
        assert rate == (100.0 + 200.0) / 2.0    # all ranks' units over that time
        assert sorted(insts) == [0, 1]          # distinct replicas



def test_single_process_defaults():
    assert RP.max_over_ranks(3.5) == 3.5
    assert RP.aggregate_rate(10.0, 2.0) == 5.0
