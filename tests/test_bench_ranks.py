"""The multi-GPU path of bench.py, on CPU: two gloo ranks (127.0.0.1).

Replicas share no data; the only cross-rank steps are the barriers around the
timed region and the max-over-ranks time.  Each rank feeds a different local
time; both must see the maximum, and the whole-job value must count both
ranks' work against the slowest rank's time.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 150.0][rank]
    dist.barrier()
    ms = bench.reduce_max_ms(local_ms, world)
    dist.barrier()
    out[rank] = (ms, bench.whole_job_gflops(1e9, world, ms))
    dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_value():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    assert out[0][0] == out[1][0] == 150.0
    # 2 ranks x 1 GFLOP each in 150 ms
    assert out[0][1] == pytest.approx(2e9 / 0.150 / 1e9)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max_ms(12.5, 1) == 12.5
    assert bench.whole_job_gflops(2e9, 1, 1000.0) == pytest.approx(2.0)


def test_end_to_end_call_order_takes_each_call_once():
    """The end-to-end leg alternates between the smallest and the largest orders: every call
    appears exactly once, the first two are the two ends, and the order is deterministic."""
    import bench
    for n in range(0, 9):
        items = list(range(n))
        out = bench.ends_inward(items)
        assert sorted(out) == items
        if n >= 2:
            assert out[:2] == [0, n - 1]
    assert bench.ends_inward(list("abcde")) == list("aebdc")
