"""bench.py's multi-GPU form: one process per GPU, each solving its own
sources (replicas -- the solve has no exchange step, so no collective touches
the data path); only the whole-job numbers are combined: the step time is the
slowest rank's, the work and the end-to-end throughput are summed.  Run here
with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        import bench
        ms, flops, value = bench.whole_job(dist, [10.0, 12.5][rank], [1e9, 3e9][rank], "cpu")
        e2e = bench.sum_over_ranks(dist, [100.0, 50.0][rank], "cpu")
        none = bench.sum_over_ranks(dist, None, "cpu")
        q.put((rank, ms, flops, value, e2e, none))
    finally:
        dist.destroy_process_group()


def test_whole_job_over_two_gloo_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, flops, value, e2e, none in out:
        assert ms == 12.5 and flops == 4e9
        assert value == pytest.approx(4e9 / 12.5e-3 / 1e9)
        assert e2e == 150.0 and none is None


def test_single_process_is_its_own_whole_job():
    import bench
    assert bench.whole_job(None, 20.0, 2e9, "cpu") == (20.0, 2e9, pytest.approx(100.0))
    assert bench.sum_over_ranks(None, 5.0, "cpu") == 5.0
