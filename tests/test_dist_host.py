"""The multi-rank path of bench.py on the host (gloo, world size 2, no GPU):
the ranks' source sets are disjoint and equally sized, the timing
reductions take the slowest rank's time and the sum of the ranks'
visibilities (the whole-job value), and the final reduce-sum of the ranks'
partial cubes gives the cube of the whole source set (each rank stacks its
share of the windows; the oracle stands in for the GPU on the host)."""
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


def _rank_cubes(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import numpy as np
    import torch
    import torch.distributed as dist

    import bench
    from oracle import oracle as O
    from paper_2609_01897_gb300 import synth
    w, r, _ = bench.dist_setup(None, backend="gloo")
    try:
        wl = synth.tiny("cpu")
        f0, df = O.auto_lattice([s.freqs for s in wl.spws], [s.z for s in wl.spws], wl.nrest, wl.central_freq)
        cube = O.make_cube(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, f0, df, 0, 0)
        mine = [s for i, s in enumerate(wl.spws) if i % w == r]      # this rank's windows
        src = [O.Source(s.uvw.numpy(), s.freqs, s.vis.numpy(), s.weights.numpy(), s.flags.numpy(), s.l, s.m, s.z)
               for s in mine]
        part = O.stack(cube, src, nthreads=2)
        t = {"sum_wv": torch.view_as_real(torch.from_numpy(part["sum_wv"])).contiguous(),
             "sum_w": torch.from_numpy(part["sum_w"]), "sum_wvv": torch.from_numpy(part["sum_wvv"]),
             "count": torch.from_numpy(part["count"].astype(np.int64))}
        total = bench.reduce_cubes(w, t)
        if r == 0:
            q.put({k: v.numpy() for k, v in total.items()})
        bench.barrier(w)
    finally:
        dist.destroy_process_group()


def test_two_ranks_partial_cubes_reduce_to_the_whole_stack(oracle_mod):
    import numpy as np
    from paper_2609_01897_gb300 import synth
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_cubes, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    O = oracle_mod
    wl = synth.tiny("cpu")
    f0, df = O.auto_lattice([s.freqs for s in wl.spws], [s.z for s in wl.spws], wl.nrest, wl.central_freq)
    cube = O.make_cube(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, f0, df, 0, 0)
    src = [O.Source(s.uvw.numpy(), s.freqs, s.vis.numpy(), s.weights.numpy(), s.flags.numpy(), s.l, s.m, s.z)
           for s in wl.spws]
    whole = O.stack(cube, src, nthreads=2)
    np.testing.assert_array_equal(got["count"], whole["count"].astype(np.int64))
    assert got["count"].sum() > 0
    np.testing.assert_allclose(got["sum_w"], whole["sum_w"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(got["sum_wvv"], whole["sum_wvv"], rtol=1e-12, atol=1e-9)
    wv = got["sum_wv"][..., 0] + 1j * got["sum_wv"][..., 1]
    np.testing.assert_allclose(wv, whole["sum_wv"], rtol=1e-12, atol=1e-9)
