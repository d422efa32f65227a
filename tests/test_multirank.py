"""The N > 1 path of bench.py on CPU with two gloo ranks: every rank runs the same solve (replicas, no
collective on the data path); the reported time is the largest over the ranks, taken after a
barrier; only rank 0 prints, and the reference arm runs on rank 0 alone."""
import os
import socket
import sys
import types

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    v = bench.max_over_ranks(1.0 + 0.25 * rank, world, "cpu")
    w = bench.max_over_ranks(3.0 - rank, world, "cpu")
    dist.barrier()
    q.put((rank, v, w))
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 1.25, 3.0), (1, 1.25, 3.0)]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1, "cpu") == 2.5


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    args = types.SimpleNamespace(workload="stencil_8x8x8x8", steps=1, warmup=0, gpus=2)
    bench.run_reference(args, rank=1, world=2)       # returns before any oracle work
    assert capsys.readouterr().out == ""


def test_reference_arm_of_the_largest_workload_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    args = types.SimpleNamespace(workload=bench.HEADLINE, steps=1, warmup=0, gpus=2)
    bench.run_reference_headline(args, rank=1, world=2)   # returns before any oracle work
    assert capsys.readouterr().out == ""
