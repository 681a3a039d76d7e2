"""The multi-GPU path of bench.py is replicas with no data-path collective;
its host-side aggregation (total work over ranks, max time over ranks) is
checked here with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    work, secs = bench.aggregate(100.0 * (rank + 1), 0.5 + rank, world)
    bench.barrier(world)
    q.put((rank, work, secs))
    dist.destroy_process_group()


@pytest.mark.skipif(torch.cuda.is_available(), reason="CPU gloo test")
def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, work, secs in res:
        assert work == 300.0      # 100 + 200: total work over ranks
        assert secs == 1.5        # max(0.5, 1.5): slowest rank's time


def test_aggregate_single_rank():
    import bench
    assert bench.aggregate(5.0, 2.0, 1) == (5.0, 2.0)


def test_clock_records_the_timing_rules_reject():
    """bench.py measures once more when the clock record shows a hardware
    or thermal slowdown or an SM clock stuck well below its maximum; a
    power cap alone is kept."""
    import bench
    assert not bench.bad_clocks(None)
    assert not bench.bad_clocks({"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"]})
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.bad_clocks({"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [r]})
    assert bench.bad_clocks({"sm_mhz": 1200.0, "sm_max_mhz": 2070.0, "reasons": []})
