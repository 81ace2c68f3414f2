"""The multi-GPU form of the benchmark is independent replicas (no data-path collective):
each rank advances its own grid; the ranks meet only in the barriers around the timed region
and in the reductions of the timing (max over ranks) and of the work (sum over ranks).  This
runs those host-side pieces as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank: int, world: int, port: int, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "NS3D_BENCH_GLOO": "1"})
    import bench
    w, r, local = bench.dist_init()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    t_max = bench.max_over_ranks(10.0 + rank, w)       # e.g. each rank's elapsed time
    units = bench.sum_over_ranks(1000.0 * (rank + 1), w)  # each rank's grid points x RHS
    bench.barrier(w)
    out.put((rank, t_max, units))
    dist.destroy_process_group()


def test_two_replica_ranks_reduce_time_and_work():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, units in res:
        assert t_max == 11.0          # the slowest rank sets the time
        assert units == 3000.0        # whole-job work = sum over ranks


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    """Under torchrun the oracle arm runs on rank 0 only; the other ranks return at once."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    called = []
    monkeypatch.setattr(bench, "cpu_oracle_sample", lambda *a, **k: called.append(1))
    ns = type("A", (), {"n": 8, "steps": 1, "warmup": 0, "gpus": 2, "cfl": 0.4})()
    bench.run_reference(ns, 2, 1)
    assert called == [] and capsys.readouterr().out == ""
