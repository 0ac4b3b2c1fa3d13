"""The multi-rank path of bench.py on the host (gloo, world size 2, no GPU):
the ranks' source sets are disjoint and equally sized, and the timing
reductions take the slowest rank's time and the sum of the ranks'
visibilities (the whole-job value)."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_setup(None, backend="gloo")
    try:
        ids = list(bench.shard_ids(64, r))
        allids = [None] * w
        dist.all_gather_object(allids, ids)
        slowest = bench.allmax(w, 1.5 + r)
        total = bench.allsum(w, 10.0 * (r + 1))
        bench.barrier(w)
        q.put((r, w, allids, slowest, total, dist.get_backend()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(o[0] for o in out) == [0, 1]
    for _, w, allids, slowest, total, backend in out:
        assert w == 2 and backend == "gloo"
        assert slowest == 2.5 and total == 30.0
        a, b = set(allids[0]), set(allids[1])
        assert len(a) == len(b) == 64 and not (a & b)
