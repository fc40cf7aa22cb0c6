"""The multi-rank path of bench.py on CPU.  The method's units are independent,
so N GPUs run N replicas with no collective on the data path; the only
cross-rank steps are the barriers around the timed region and the maximum of
the ranks' times.  Two gloo ranks check that step and the job throughput; the
reference arm returns at once on every rank but 0."""
import argparse
import os
import socket

import pytest

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, ms_by_rank, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms = bench.max_over_ranks(ms_by_rank[rank], dist, "cpu")
    out.put((rank, ms, bench.job_throughput(world, 10, 505, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, [10.0, 12.5], out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in got:
        assert ms == 12.5
        assert value == pytest.approx(2 * 10 * 505 / 12.5e-3)


def test_single_process_keeps_its_own_time():
    assert bench.max_over_ranks(7.0, None, "cpu") == 7.0
    assert bench.job_throughput(1, 4, 100, 8.0) == pytest.approx(4 * 100 / 8e-3)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(workload="mixed_ecc", steps=1, warmup=0, gpus=2, refine=None)
    assert bench.run_reference(args) == 0
