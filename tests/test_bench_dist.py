"""The benchmark's multi-process path on CPU (gloo, world size 2): the whole-job time is
the max over ranks, the work is the sum over ranks, and the reference arm leaves
non-zero ranks idle."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.dist_init(world)
    secs, units = bench.aggregate(1.0 + rank, 10.0 * (rank + 1), d)
    d.barrier()
    d.destroy_process_group()
    q.put((rank, secs, units))


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, secs, units in res:
        assert secs == 2.0      # max over ranks of the timed duration
        assert units == 30.0    # sum over ranks of the work


def test_reference_arm_leaves_other_ranks_idle(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(bench.parse_args(["--impl", "reference"])) == 0
