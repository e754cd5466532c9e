"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas only; the
single-field factorisation does not shard).  The per-rank timings combine as
their maximum, the whole-job rate counts every rank's evaluations, and a
batched workload splits into disjoint contiguous task ranges."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist, r, w = bench._dist("gloo")
    ms = bench.reduce_max(dist, [100.0 + 50.0 * r, 7.0 - r])
    lo, hi = bench.shard(10, r, w)
    q.put((r, w, ms, (lo, hi)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_disjoint_shards():
    torch = pytest.importorskip("torch")
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2, 2]
    for r in res:
        assert r[2] == [150.0, 7.0]              # max over ranks, on every rank
    assert res[0][3] == (0, 5) and res[1][3] == (5, 10)
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(2, 48, 150.0) == 2 * 48 / 0.15
    cover = [i for k in range(3) for i in range(*bench.shard(11, k, 3))]
    assert cover == list(range(11))
