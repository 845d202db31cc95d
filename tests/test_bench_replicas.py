"""The N > 1 path of bench.py runs independent replicas; its only
cross-rank step is the job time (max over ranks) and the whole-job value.
Checked with two gloo ranks on CPU."""
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


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    elapsed = [1.25, 2.5][rank]
    t = bench.job_seconds(elapsed, ws)
    v = bench.job_value(100.0, ws, t)
    out[rank] = (t, v)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_job_time_and_value():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(ws, port, out), nprocs=ws, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1] == (2.5, 2 * 100.0 / 2.5)


def test_single_rank_passes_time_through():
    import bench
    assert bench.job_seconds(3.0, 1) == 3.0
    assert bench.job_value(10.0, 1, 2.0) == 5.0
