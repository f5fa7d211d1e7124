"""The multi-process path of bench.py without a GPU: two gloo ranks on the
host.  Every rank decodes its own replica (no collective on the data path);
the only exchange is the timing reduction, which must return the slowest
rank's times on every rank, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 5.0], dist, "cpu")
        keys, dates = bench.make_workload(1 + rank, rows=4096)
        q.put((rank, got, int(keys[-1]), int(dates.astype("int64").sum())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_own_replicas():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, got, _, _ in res:
        assert got == [2.0, 10.0, 5.0], rank
    assert res[0][2:] != res[1][2:]            # each rank has its own data
    assert bench.whole_job_gbs(2 * 3e9, 2.0) == pytest.approx(3000.0)


def test_single_process_reduction_is_identity():
    assert bench.max_over_ranks([3, 1.5], None, "cpu") == [3.0, 1.5]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    called = []
    monkeypatch.setattr(bench, "run_reference", lambda *a, **k: called.append(a))
    bench.main()
    assert not called and capsys.readouterr().out == ""
