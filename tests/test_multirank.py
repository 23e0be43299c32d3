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
