"""The multi-rank path of bench.py on CPU: world size 2 over gloo (no GPU).

Every rank runs an independent replica of the lattice (the step needs no
exchange), so the only cross-rank operations are the barrier and the max of
the timings; the whole-job value counts the updates of all replicas."""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [12.5, 17.25][rank]
    ms = bench.reduce_max(local_ms, "cpu")
    value = bench.whole_job_glups(world, 4096 * 4096, 100, ms)
    dist.barrier()
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expected = 2 * 4096 * 4096 * 100 / (17.25e-3) / 1e9
    for rank, ms, value in out:
        assert ms == 17.25
        assert value == pytest.approx(expected, rel=1e-12, abs=0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench

    class A:
        size, steps, warmup, gpus = 256, 3, 1, 2
    bench.run_reference(A, ws=2, rank=1)
    assert capsys.readouterr().out == ""
    bench.run_reference(A, ws=2, rank=0)
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["unit"] == "GLUPS" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
