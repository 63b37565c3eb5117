"""Several GPUs run the benchmark as independent replicas: each rank evolves its own circuit, and
the ranks meet only to take the slowest rank's time (no collective on the data path).  That host
logic on two gloo ranks on the CPU: every rank sees the largest time, the whole-job rate counts
all ranks' gates over it, and the reference arm prints on rank 0 only."""

import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    ms = bench.max_over_ranks(40.0 + 10.0 * rank, dist, "cpu")  # rank 1 is the slow one
    e2e = bench.max_over_ranks(0.05 - 0.01 * rank, dist, "cpu")  # rank 0 is the slow one
    out.put((r, w, ms, e2e, bench.replica_rate(bench.N_GATES, 3, w, ms / 1e3)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert all(x[2] == 50.0 and x[3] == 0.05 for x in res)
    assert all(abs(x[4] - 1000 * 3 * 2 / 0.050) < 1e-6 for x in res)


def test_one_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.replica_rate(1000, 5, 1, 0.25) == 20000.0


def test_reference_arm_prints_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.run_reference(bench.parse_args())  # rank 1 returns at once: no oracle work, no line
    assert capsys.readouterr().out == ""
