"""The multi-GPU path of bench.py is independent replicas (no collective on
the data path): its host logic, two ranks over gloo on the CPU."""
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = [7.5, 9.25][rank]                      # the ranks' own step times
        m = bench.max_over_ranks(ms, world, "cpu")
        q.put((rank, m, bench.replica_seconds_per_svd(m, world)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_step():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slower rank's time; 2 SVDs per 9.25 ms step
    assert [o[1] for o in out] == [9.25, 9.25]
    assert all(abs(o[2] - 9.25e-3 / 2) < 1e-15 for o in out)


def test_single_rank_is_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1, None) == 3.0
    assert bench.replica_seconds_per_svd(3.0, 1) == 3.0e-3


def test_reference_arm_prints_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    a = types.SimpleNamespace(warmup=3, steps=1, n=16384, kind="uniform", seed=0, gpus=2)
    bench.run_reference(a, rank=1, world=2)     # returns before any work
    assert capsys.readouterr().out == ""
