"""The multi-process path of the benchmark on CPU (gloo, world size 2): every
rank gets the slowest rank's time, and the whole-job figure counts the frames
of all ranks over that time.  The GPU path has no exchange step (independent
replicas), so this reduction is the only cross-rank operation."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, times, out):
    import torch
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    dist.barrier()
    m = bench.max_over_ranks(times[rank], torch.device("cpu"), ws)
    v = bench.whole_job_mpix(10 * ws, 512 * 512, m)
    out[rank] = (m, v)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    ws = 2
    times = [12.5, 17.25]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(ws, _free_port(), times, out), nprocs=ws, join=True,
                       start_method="spawn")
    for r in range(ws):
        m, v = out[r]
        assert m == max(times)
        assert v == pytest.approx(10 * ws * 512 * 512 / (max(times) / 1e3) / 1e6)


def test_single_process_is_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(3.5, None, 1) == 3.5
    assert bench.whole_job_mpix(20, 512 * 512, 1000.0) == pytest.approx(20 * 512 * 512 / 1e6)


def _failing_rank_main(rank, ws, port, out):
    import time
    import torch
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)                 # as torchrun sets them
    os.environ["WORLD_SIZE"] = str(ws)
    bench.init_replicas("gloo", timeout_s=10.0)
    if rank == 1:
        os._exit(0)                      # a replica that dies between steps, before the reduction
    t0 = time.perf_counter()
    try:
        bench.max_over_ranks(5.0, torch.device("cpu"), ws)
        out["raised"] = False
    except Exception as e:               # the survivor learns of it as an error, not a hang
        out["raised"] = True
        out["what"] = type(e).__name__
    out["seconds"] = time.perf_counter() - t0


def test_dead_replica_is_an_error_not_a_hang():
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_failing_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True,
                       start_method="spawn")
    assert out["raised"] is True, dict(out)
    assert out["seconds"] < 60.0
