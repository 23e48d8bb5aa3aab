"""The benchmark's multi-rank path on CPU: two gloo ranks on 127.0.0.1.

bench.py runs one independent controller replica per GPU (the step has no
exchange between replicas); the ranks meet only at the barriers around the
timed region and in the maximum over ranks of the step time, and the
reported value is all ranks' sample-steps divided by that maximum.  The
reference arm runs on rank 0 alone."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    got_ws, got_rank, _ = bench.dist_setup()
    bench.barrier(got_ws)
    ms = bench.allmax(got_ws, 1.0 + rank)  # rank r "took" 1 + r ms
    bench.barrier(got_ws)

    class Args:
        workload, ref_samples, warmup, steps, gpus = "unicycle_small", 4, 0, 1, ws

    printed = None
    if rank != 0:
        printed = bench.run_reference(Args, got_ws, got_rank)
    out[rank] = (got_ws, got_rank, ms, printed)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0][:3] == (2, 0, 2.0)
    assert res[1][:3] == (2, 1, 2.0)
    assert res[1][3] is None  # the reference arm does no work off rank 0
    # whole-job value: both replicas' sample-steps over the slowest rank's time
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_value(ws, 4096 * 50, res[0][2]) == pytest.approx(2 * 4096 * 50 / 2.0e-3)
