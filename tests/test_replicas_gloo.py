"""The N > 1 path (independent replicas, max-over-ranks timing) with two gloo
ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2010_00409_gb300 import replicas as R


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = R.env()
        units = R.units_for_rank(64, w, r)
        my_time = 1.0 + 0.5 * r                       # rank 1 is the slowest
        R.barrier()
        t_max = R.max_over_ranks(my_time)
        rate = R.whole_job_rate(len(units), w, t_max)
        q.put((r, units, t_max, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_units_and_agree_on_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    units0, units1 = res[0][1], res[1][1]
    assert sorted(units0 + units1) == list(range(64)) and not set(units0) & set(units1)
    assert res[0][2] == res[1][2] == 1.5
    assert res[0][3] == res[1][3] == pytest.approx(32 * 2 / 1.5)


def test_single_process_helpers():
    assert R.units_for_rank(5, 1, 0) == [0, 1, 2, 3, 4]
    assert R.max_over_ranks(3.0) == 3.0
    with pytest.raises(ValueError):
        R.units_for_rank(5, 2, 2)
    with pytest.raises(ValueError):
        R.whole_job_rate(1.0, 1, 0.0)
