"""The multi-process path of bench.py on the CPU: two ranks (gloo, 127.0.0.1) run
bench.Replicas exactly as the torchrun replicas do on the GPUs (NCCL there).  The replicas
share no data; the process group only brackets the timed region with barriers and combines
the per-rank figures (the max of the times, the sum of the work), so the JSON line's value is
the whole job's work over the slowest rank."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    reps = bench.Replicas("gloo")
    try:
        out = {"rank": reps.rank, "world": reps.world, "local": reps.local}
        reps.barrier()
        out["max"] = reps.max(10.0 * (rank + 1))          # per-rank times 10, 20
        out["sum"] = reps.sum(rank + 1.0)                 # per-rank work 1, 2
        # the whole-job value a rank would print: the work of all ranks over the slowest rank
        ms = reps.max(5.0 + rank)
        out["value"] = reps.sum(100.0) / ms
        reps.barrier()
        q.put(out)
    finally:
        reps.close()


def test_two_replicas_combine_times_and_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    outs = []
    try:
        for _ in range(2):
            outs.append(q.get(timeout=120))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    outs.sort(key=lambda o: o["rank"])
    assert [o["rank"] for o in outs] == [0, 1]
    for o in outs:
        assert o["world"] == 2 and o["local"] == o["rank"]
        assert o["max"] == 20.0
        assert o["sum"] == 3.0
        assert o["value"] == pytest.approx(200.0 / 6.0)


def test_one_replica_needs_no_process_group(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    sys.path.insert(0, ROOT)
    import bench
    reps = bench.Replicas("gloo")
    assert (reps.rank, reps.world, reps.local) == (0, 1, 0) and reps.dist is None
    reps.barrier()
    assert reps.max(3.5) == 3.5 and reps.sum(2.0) == 2.0
    reps.close()
