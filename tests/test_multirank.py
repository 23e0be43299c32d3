"""The N > 1 host logic of bench.py on CPU: two gloo ranks, each timing its
own replica, report the units of both ranks over the slower rank's time
(weak scaling, replicas only), and each rank draws a different replica."""
import os
import socket
import sys

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
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2204_14167_gb300 import synth
    ws, r, _ = bench._dist()
    units = 100.0 * (rank + 1)
    t_ms = 10.0 * (rank + 1)
    rate, tmax = bench.whole_job_rate(units, t_ms, dist, "cpu")
    pos, _, _ = synth.ions((16, 8, 16), 4, 4, 20220430 + r, 1.0, 0.0)
    out[rank] = (ws, r, rate, tmax, float(pos.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (ws, r, rate, tmax, _) in res.items():
        assert ws == 2 and r == rank
        assert tmax == 20.0                       # the slower rank
        assert rate == pytest.approx(300.0 / 20e-3)
    assert res[0][4] != res[1][4]                 # each rank draws its own replica


def test_single_process_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(500.0, 10.0) == (50000.0, 10.0)


def test_clock_samples_summary():
    """The clock record of a bench line: median SM clock of the sampled GPU
    only, its maximum clock, and every throttle reason seen active."""
    sys.path.insert(0, ROOT)
    import bench
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1, 1200, 2070, 300.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1010.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    c = bench.parse_clocks(lines, 0)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.parse_clocks(lines, 1)["reasons"] == ["hw_slowdown"]
    assert bench.parse_clocks(lines, 3) is None
