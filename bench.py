#!/usr/bin/env python
"""Stacked visibilities per second on GB300 (ViSta hot path, libvista).

One step = one full stacking pass: queue every (source, window) of the
workload, vista_run (the cube is zeroed once and accumulates across steps).
The default workload is the batched uneven stack (2000 sources, lognormal
row counts, 1-4 windows of 128-3840 channels, 2 or 4 pols, one persistent
launch per class replayed from a CUDA graph; cube 256 x 256 uv cells x 1024
rest channels x 4 pols).  Its ~1.7 TB of in-cube inputs per step are views
into a 96 GB device pool, resident in HBM before the timed region and far
larger than L2, so no L2 flush is needed between steps.  --config
alma_compact, mixed, wideband_hi and tiny select the other workloads.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores instead, on bounded samples of the same workload.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torchrun, one rank per GPU, each stacking its own 64 sources (weak scaling,
no collective on the data path).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "stacked vis/s and % HBM roofline, mixed+batched vs plain FP64 GPU, <=1e-5 rel err"
UNIT = "vis/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", default="batched", choices=["alma_compact", "tiny", "wideband_hi", "batched", "mixed"])
    p.add_argument("--reproject", action="store_true",
                   help="full re-projection of Eq. 1: every window names its phase centre and stacking position")
    p.add_argument("--storage", default="c64", choices=["c64", "f16", "bf16"],
                   help="visibility storage (16-bit: one power-of-two scale per window)")
    p.add_argument("--pool-gb", type=float, default=96.0, help="batched: device pool the windows alias (GB)")
    p.add_argument("--sources", type=int, default=0, help="sources per rank (0 = the workload's own)")
    p.add_argument("--nrest", type=int, default=0,
                   help="batched: rest channels of the cube (0 = 1024; fewer gives a smaller cube for captures)")
    p.add_argument("--fp64-steps", type=int, default=1, help="timed steps of the plain FP64 leg (0 = skip)")
    p.add_argument("--e2e-steps", type=int, default=4, help="timed host-memory steps (0 = skip)")
    p.add_argument("--e2e-readback", choices=["sparse", "dense"], default="sparse",
                   help="what each end-to-end step reads back: the touched cube entries (index and sums) or "
                        "the whole cube")
    p.add_argument("--e2e-gb", type=float, default=24.0,
                   help="pinned host memory for the end-to-end leg: windows are taken in order while their "
                        "host copies fit (GB)")
    p.add_argument("--cpu-sample", type=int, default=40,
                   help="windows timed once in the oracle baseline of our arm (0 = skip)")
    p.add_argument("--cpu-gb", type=float, default=56.0,
                   help="host memory the oracle baseline may take: its FP64 cube (40 B per entry) plus the "
                        "sampled windows (GB); windows past it are left out, and a larger cube skips the leg")
    p.add_argument("--ref-sample", type=int, default=8, help="windows per step of the reference (oracle) arm")
    p.add_argument("--tuning", default="", help="rows,chans_per_lane,warps,sort,prefetch")
    p.add_argument("--regrid-reps", type=int, default=3,
                   help="timed calls of the per-row output (Eq. 3) on the workload's widest window (0 = skip)")
    p.add_argument("--contsub-reps", type=int, default=3,
                   help="timed calls of the continuum subtraction over the cube (0 = skip)")
    p.add_argument("--autotune", type=int, default=0,
                   help="autotune the launch shape first over this many candidates (0 = no)")
    return p.parse_args()


# ------------------------------------------------------------------ plumbing

def dist_setup(args, backend=None):
    """One process per GPU (NCCL); without CUDA, or asked for (host-side
    tests), gloo."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = backend or ("nccl" if torch.cuda.is_available() else "gloo")
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank, local


def shard_ids(n, rank):
    """Source ids of one rank: every rank stacks its own n sources (replicas,
    disjoint seeds, no exchange on the data path)."""
    return range(rank * n, rank * n + n)


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(ws, x, op):
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def allmax(ws, x):
    if ws == 1:
        return x
    import torch.distributed as dist
    return _reduce(ws, x, dist.ReduceOp.MAX)


def allsum(ws, x):
    if ws == 1:
        return x
    import torch.distributed as dist
    return _reduce(ws, x, dist.ReduceOp.SUM)


def reduce_cubes(ws, cube):
    """The one exchange step of a multi-GPU stack: the sum of the ranks'
    partial cubes on rank 0, sums in FP64 and counts as exact integers, one
    reduction per array (NCCL moves them over the GPUs' links; gloo on the
    host).  Returns rank 0's total (other ranks: their arrays, overwritten)."""
    if ws == 1:
        return cube
    import torch.distributed as dist
    out = {}
    for k, v in cube.items():
        t = v.to(torch.int64) if k == "count" else v.to(torch.float64)
        dist.reduce(t, dst=0, op=dist.ReduceOp.SUM)
        out[k] = t
    return out


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.p = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                       "-i", str(gpu_index), "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_traffic(n_vis, config):
    """DRAM bytes of a step's stacking launches from the committed ncu summary
    of this workload (profiles/stack_mixed_<config>.md), scaled by the step's
    visibilities -- or None without a summary, or once the kernel source
    differs from the one the counters were taken on."""
    import hashlib
    import re
    try:
        txt = open(os.path.join(ROOT, "profiles", "stack_mixed_%s.md" % config)).read()
        sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt).group(1)
        per_vis = float(re.search(r"traffic_bytes_per_vis:\s*([0-9.]+)", txt).group(1))
    except (OSError, AttributeError, ValueError):
        return None
    h = hashlib.sha256()
    for f in ("vista_stack.cuh", "vista_device.cuh"):
        with open(os.path.join(ROOT, "paper_2609_01897_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return per_vis * n_vis if h.hexdigest() == sha else None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ workload

def in_cube_sources(meta, nrest):
    """Rest lattice of a whole source set and the ids of the sources with a
    channel inside it (computed by the library's host planner)."""
    from paper_2609_01897_gb300 import vista as V
    f0, df = V.plan_lattice([s.freqs for s in meta.spws], [s.z for s in meta.spws], nrest, meta.central_freq)
    ids = set()
    for s in meta.spws:
        _, nb, _ = V.plan_channels(s.freqs, s.z, f0, df, nrest, V.BIN_OVERLAP)
        if (nb > 0).any():
            ids.add(s.source)
    return f0, df, sorted(ids)


def make_workload(args, rank, device):
    from paper_2609_01897_gb300 import synth
    if args.config == "tiny":
        wl = synth.tiny(device)
    elif args.config == "mixed":
        # the sources of a 64-source set whose windows reach the cube, on the
        # lattice and cell size of the whole set (the rest never add a visibility)
        n = args.sources or 64
        meta = synth.mixed("cpu", n_sources=n, src_ids=shard_ids(n, rank), meta_only=True)
        f0, df, ids = in_cube_sources(meta, meta.nrest)
        wl = synth.mixed(device, src_ids=ids, du=meta.du)
        wl.rest_f0, wl.rest_df = f0, df
    elif args.config == "wideband_hi":
        # the complex-half variant holds 48 sources (drawn directly as 16-bit pairs)
        n = args.sources or (24 if args.storage == "c64" else 48)
        ids = shard_ids(n, rank)
        wl = synth.wideband_hi(device, n_sources=n, src_ids=ids, storage=args.storage)
        return synth.with_reprojection(wl, math.radians(-30.0)) if args.reproject else wl
    else:
        n = args.sources or {"alma_compact": 64, "batched": 2000}[args.config]
        ids = shard_ids(n, rank)
        if args.config == "alma_compact":
            wl = synth.alma_compact(device, n_sources=n, src_ids=ids)
        else:
            wl = synth.batched(device, n_sources=n, src_ids=ids, pool_gb=args.pool_gb, nrest=args.nrest or 1024)
    if args.reproject:
        if args.config == "batched":
            raise SystemExit("--reproject applies to the array workloads (the batched stack has no sky geometry)")
        wl = synth.with_reprojection(wl, math.radians(-30.0))
    if args.storage != "c64":
        if args.config == "batched":
            raise SystemExit("--storage applies to workloads with their own arrays (not the aliased pool)")
        wl = synth.half_storage(wl, args.storage)
    return wl


def host_vis(s):
    """A window's visibilities as complex numpy (16-bit storage dequantised)."""
    if s.vis.dtype in (torch.float16, torch.bfloat16):
        return torch.view_as_complex(s.vis.to(torch.float32).mul_(s.vis_scale)).cpu().numpy()
    return s.vis.cpu().numpy()


def vis_bytes(v):
    return {torch.complex64: 8, torch.complex128: 16, torch.float16: 4, torch.bfloat16: 4}[v.dtype]


def algorithmic_bytes(wl, f0, df, touched):
    """Bytes a stacking pass must move at least: every visibility of a channel
    that reaches the cube (value + u8 flag), uvw + weights of every row that
    has such a channel, and one read-modify-write (2 x 20 B) per touched
    cube entry."""
    from paper_2609_01897_gb300 import vista as V
    tot_vis, tot_bytes = 0, 0
    for s in wl.spws:
        j0, nb, _ = V.plan_channels(s.freqs, s.z, f0, df, wl.nrest, V.BIN_OVERLAP)
        nin = int((nb > 0).sum())
        nrow, npol = int(s.vis.shape[0]), int(s.vis.shape[2])
        nv = nrow * nin * npol
        tot_vis += nv
        tot_bytes += nv * (vis_bytes(s.vis) + (1 if s.flags is not None else 0))
        if nin:
            tot_bytes += nrow * (24 + 4 * npol)
    tot_bytes += int(touched) * 40
    return tot_vis, tot_bytes


def one_step(st, wl, host=None):
    """One pass of the hot path over the workload: queue every window, run.
    The cube accumulates across steps (runs are additive)."""
    srcs = wl.spws if host is None else host
    for s in srcs:
        st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z, pol_map=s.pol_map,
                      vis_scale=s.vis_scale, reproject=s.radec)
    st.run()


# ------------------------------------------------------------------ our arm

def open_stack(wl, precision, tuning):
    from paper_2609_01897_gb300 import vista as V
    st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, rest_f0=wl.rest_f0, rest_df=wl.rest_df,
                 central_freq=wl.central_freq, precision=precision)
    if tuning:
        st.set_tuning(*tuning)
    return st


def timed_steps(st, wl, steps, warmup, ws, host=None, split_steps=2):
    """Time `steps` steps after `warmup` untimed ones (from the second run on,
    an unchanged source set replays its captured graph), then split a few
    more runs, launched directly with event timing, into pre-pass and
    stacking time.  Returns (ms per step, per-step split, graph runs timed)."""
    stream = torch.cuda.current_stream()
    st.zero()
    for _ in range(warmup):
        one_step(st, wl, host)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    g0 = st.graph_runs()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one_step(st, wl, host)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1) / steps
    graph_runs = st.graph_runs() - g0
    st.enable_timing(True)
    for _ in range(split_steps):
        one_step(st, wl, host)
    t = st.timing()
    st.enable_timing(False)
    t = {k: v / split_steps for k, v in t.items()}
    return ms, t, graph_runs


def windows_in_cube(wl, f0, df, n):
    """The first n windows that have channels inside the cube's rest range."""
    from paper_2609_01897_gb300 import vista as V
    out = []
    for s in wl.spws:
        _, nb, _ = V.plan_channels(s.freqs, s.z, f0, df, wl.nrest, V.BIN_OVERLAP)
        if (nb > 0).any():
            out.append(s)
        if len(out) == n:
            break
    return out


def cpu_baseline(wl, f0, df, nsample, host_gb):
    from oracle import oracle as O
    cube_b = wl.nu * wl.nv * wl.nrest * wl.npol * 40
    if cube_b > host_gb * 1e9:
        return {"skipped": "the oracle's FP64 cube would take %.0f GB of host memory (--cpu-gb %.0f)" % (
            cube_b / 1e9, host_gb)}
    srcs, used = [], cube_b
    for s in windows_in_cube(wl, f0, df, nsample):
        b = s.vis.numel() * max(8, vis_bytes(s.vis)) + s.uvw.numel() * 8 + s.weights.numel() * 4 + (
            0 if s.flags is None else s.flags.numel())
        if srcs and used + b > host_gb * 1e9:
            break
        used += b
        srcs.append(O.Source(s.uvw.cpu().numpy(), s.freqs, host_vis(s), s.weights.cpu().numpy(),
                             None if s.flags is None else s.flags.cpu().numpy(), s.l, s.m, s.z, s.pol_map,
                             radec=s.radec))
    cube = O.make_cube(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, f0, df, 0, 0)
    nthreads = os.cpu_count() or 1
    t0 = time.perf_counter()
    out = O.stack(cube, srcs, nthreads=nthreads)
    dt = time.perf_counter() - t0
    n = int(out["stats"]["n_vis"])
    return {"value": n / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": "%d of %d windows (%d visibilities), %.1f s" % (len(srcs), len(wl.spws), n, dt)}


def run_ours(args):
    from paper_2609_01897_gb300 import build as B
    from paper_2609_01897_gb300 import vista as V
    ws, rank, local = dist_setup(args)
    B.build()
    V.lib()
    tuning = tuple(int(x) for x in args.tuning.split(",")) if args.tuning else None
    wl = make_workload(args, rank, "cuda")
    torch.cuda.synchronize()

    # mixed-precision path (the headline)
    st = open_stack(wl, V.PREC_MIXED, tuning)
    if args.autotune > 0:
        for s in wl.spws:
            st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z, pol_map=s.pol_map,
                          vis_scale=s.vis_scale, reproject=s.radec)
        st.autotune(budget=args.autotune, reps=1)
        st.run()                       # the queue the autotuner left in place: the first run
    else:
        one_step(st, wl)
    eff_tuning = st.tuning()
    f0, df = st.lattice()
    cnt = st.read_cube(which=("count",))["count"]
    touched = int((cnt > 0).sum())
    del cnt
    stats = st.stats()
    n_vis, alg = algorithmic_bytes(wl, f0, df, touched)
    assert n_vis == stats["n_vis"], (n_vis, stats)
    clk = Clocks(local)
    ms, tm, graph_runs = timed_steps(st, wl, args.steps, args.warmup, ws)
    clocks = clk.stop()
    red_per_vis = stats["n_reductions"] / max(1, n_vis)   # of the first run
    ms_max = allmax(ws, ms)
    n_vis_all = allsum(ws, n_vis)   # every rank's visibilities (the ranks' source sets differ)
    value = n_vis_all / (ms_max * 1e-3)
    stack_ms = tm["stack_ms"]
    peak, peak_kind = measured_peaks()
    achieved = alg / (stack_ms * 1e-3) / 1e9 if stack_ms > 0 else 0.0
    launches = int(round(tm["launches"])) * args.steps
    # end to end through the C ABI with host buffers, straight after the timed
    # steps (after the other legs the same steps have taken up to twice as
    # long on this shared machine); where its stack does not fit beside the
    # main one, again once the main stack is closed (below)
    e2e, e2e_retry = None, False
    if args.e2e_steps > 0:
        try:
            e2e = run_e2e(args, wl, tuning, f0, df, ws)
        except (RuntimeError, MemoryError) as exc:
            e2e, e2e_retry = {"error": str(exc)[:200]}, True
    link = host_link_peak() if rank == 0 and args.e2e_steps > 0 else None
    regrid = time_regrid(st, wl, f0, df, args.regrid_reps, peak) if args.regrid_reps > 0 else None
    contsub = time_contsub(st, wl, args.contsub_reps, peak) if args.contsub_reps > 0 else None
    # several GPUs: the final reduce-sum of the partial cubes into rank 0 (after the timed region)
    cube_reduce_ms = None
    if ws > 1:
        import torch.distributed as dist
        on_dev = dist.get_backend() == "nccl"
        part = st.read_cube(device=on_dev, f64=True)
        barrier(ws)
        t0 = time.perf_counter()
        total = reduce_cubes(ws, part)
        if on_dev:
            torch.cuda.synchronize()
        cube_reduce_ms = allmax(ws, (time.perf_counter() - t0) * 1e3)
        del part, total
    st.close()
    if e2e_retry:
        torch.cuda.empty_cache()
        try:
            e2e = run_e2e(args, wl, tuning, f0, df, ws)
            e2e["order"] = "after the main stack was closed (both stacks did not fit on the device)"
        except (RuntimeError, MemoryError) as exc:
            e2e = {"error": str(exc)[:200]}


    # plain FP64 GPU form on the same inputs
    fp64 = None
    if args.fp64_steps > 0:
        st64 = open_stack(wl, V.PREC_FP64, None)
        ms64, _, _ = timed_steps(st64, wl, args.fp64_steps, 1, ws, split_steps=1)
        st64.close()
        ms64 = allmax(ws, ms64)
        fp64 = {"value": n_vis_all / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                "speedup_mixed_vs_fp64": ms64 / ms_max}

    cpu = None
    if rank == 0 and ws == 1 and args.cpu_sample > 0:
        cpu = cpu_baseline(wl, f0, df, args.cpu_sample, args.cpu_gb)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (FP64 geometry, tables, seeds)", "data": "synthetic",
            "config": {"workload": workload_name(wl), "n_vis_per_step": n_vis, "touched_cube_entries": touched,
                       "l2_flush": "none needed: ~%.0f GB of inputs per step, L2 is 0.13 GB" % (alg / 1e9),
                       "tuning": st_tuning_str(eff_tuning),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": measured_traffic(n_vis, args.config), "kernel": "stack_mixed",
                         "algorithmic_bytes_per_launch": alg, "kernel_ms": stack_ms,
                         "peak_source": peak_kind},
            "prepass_ms": tm["prepass_ms"],
            "cube_reduce_ms": cube_reduce_ms,
            "graph_replays_timed": graph_runs,
            "cube_reductions_per_vis": red_per_vis,
            "fp64_gpu": fp64,
            "regrid_rows": regrid,
            "contsub": contsub,
            "e2e": e2e,
            "host_link": link,
            "cpu_baseline": cpu,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def time_regrid(st, wl, f0, df, reps, peak):
    """The paper's per-row output (Eq. 3, vista_regrid_rows) on the workload's
    widest window that reaches the cube: rows/s and the kernel's bytes (every
    (row, channel, pol) value and flag of the window read once, the uvw, and
    the [nrow][nrest][npol] outputs written: 8 + 4 B each) per second."""
    from paper_2609_01897_gb300 import vista as V
    best = None
    for s in wl.spws:
        _, nb, _ = V.plan_channels(s.freqs, s.z, f0, df, wl.nrest, V.BIN_OVERLAP)
        if (nb > 0).any() and s.vis.shape[0] > 0 and (best is None or s.vis.shape[1] > best.vis.shape[1]):
            best = s
    if best is None:
        return None
    s = best
    nrow, nchan, npol = (int(x) for x in s.vis.shape[:3])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the outputs are allocated once (warm-up call) and written in place by every timed call
    ov, ow, _ = st.regrid_rows(s.uvw, s.freqs, s.vis, s.flags, l=s.l, m=s.m, z=s.z, vis_scale=s.vis_scale)
    out = (torch.view_as_real(ov), ow)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0.record(stream)
    for _ in range(reps):
        st.regrid_rows(s.uvw, s.freqs, s.vis, s.flags, l=s.l, m=s.m, z=s.z, vis_scale=s.vis_scale, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del out, ov, ow
    nbytes = nrow * nchan * npol * (vis_bytes(s.vis) + (1 if s.flags is not None else 0)) + nrow * 24 + \
        nrow * wl.nrest * npol * 12
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"window": "%d rows x %d ch x %d pol onto %d rest channels" % (nrow, nchan, npol, wl.nrest),
            "ms": ms, "rows_per_s": nrow / (ms * 1e-3), "gb_s": gbs, "frac_hbm": gbs / peak,
            "bytes_per_call": int(nbytes)}


def time_contsub(st, wl, reps, peak):
    """Continuum subtraction over the cube (vista_contsub, order 1, the
    central eighth of the rest channels marked as line): ms per call and the
    bytes of one pass over the cube's sums (the FP32 part and the FP64
    master: 16 + 32 B per entry) plus the output (8 B per entry)."""
    nrest = wl.nrest
    free = np.ones(nrest, dtype=bool)
    free[nrest // 2 - nrest // 16: nrest // 2 + nrest // 16] = False
    out = st.contsub(free, 1)      # warm (the output buffer is reused)
    t = []
    for _ in range(reps):
        t0 = time.perf_counter()
        st.contsub(free, 1, out=out)
        t.append(time.perf_counter() - t0)
    ms = 1e3 * min(t)
    n = wl.nu * wl.nv * nrest * wl.npol
    nbytes = n * (16 + 32 + 8)
    gbs = nbytes / (ms * 1e-3) / 1e9
    del out
    return {"order": 1, "ms": ms, "entries": n, "gb_s": gbs, "frac_hbm": gbs / peak, "bytes_per_call": nbytes,
            "timing": "host clock around the synchronous call (includes the stream sync and error-word read)"}


def to_pinned(t):
    if t is None:
        return None
    out = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
    out.copy_(t)
    return out


def window_io(s, f0, df, nrest):
    """(in-cube visibilities, the least bytes a host copy of one window needs):
    uvw and weights of every row, and the channels read (the in-cube range
    rounded out to whole flag words) of vis and flags.  vista_run may copy
    more (whole flag rows); the e2e figure reports what it copied."""
    from paper_2609_01897_gb300 import vista as V
    _, nb, _ = V.plan_channels(s.freqs, s.z, f0, df, nrest, V.BIN_OVERLAP)
    nrow, nch, npol = (int(x) for x in s.vis.shape[:3])
    ks = np.nonzero(nb > 0)[0]
    if ks.size == 0 or nrow == 0:
        return 0, 0
    al = 1 if npol >= 4 else 4 // npol
    lo, hi = int(ks[0]) // al * al, min(nch, (int(ks[-1]) + 1 + al - 1) // al * al)
    nin = hi - lo
    h2d = nrow * (24 + 4 * npol) + nrow * nin * npol * vis_bytes(s.vis)
    if s.flags is not None:
        h2d += nrow * ((nin * npol + 3) // 4 * 4)
    npm = npol if s.pol_map is None else int((np.asarray(s.pol_map) >= 0).sum())
    return nrow * int(ks.size) * npm, h2d


def run_e2e(args, wl, tuning, f0, df, ws):
    """Same metric through the public API with pinned HOST buffers: every step
    copies its inputs host->device (inside vista_run) and reads the cube back
    to host memory (by default its touched entries, vista_read_cube_sparse;
    --e2e-readback dense: the whole cube, overlapping the next step).  The
    windows are taken in order while their pinned host
    copies fit in --e2e-gb (all of them for the array workloads; for the
    batched stack, whose windows are views into a device pool, a stated
    leading subset)."""
    from paper_2609_01897_gb300 import synth
    from paper_2609_01897_gb300 import vista as V
    host, h2d, n_vis, pinned = [], 0, 0, 0
    for s in wl.spws:
        nv, hb = window_io(s, f0, df, wl.nrest)
        if nv == 0:
            continue
        size = sum(t.numel() * t.element_size() for t in (s.uvw, s.vis, s.weights, s.flags) if t is not None)
        if pinned + size > args.e2e_gb * 1e9:
            break
        pinned += size
        host.append(synth.SourceSpw(to_pinned(s.uvw), s.freqs, to_pinned(s.vis), to_pinned(s.weights),
                                    to_pinned(s.flags), s.l, s.m, s.z, s.pol_map, s.source, s.vis_scale, s.radec))
        n_vis += nv
        h2d += hb
    if not host:
        return {"error": "no window fits in --e2e-gb"}
    sub = synth.Workload(wl.name, wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, wl.central_freq, host,
                         df, f0)
    ste = open_stack(sub, V.PREC_MIXED, tuning)
    sparse = args.e2e_readback == "sparse"
    try:
        outs, t0 = None, 0.0
        split = {"queue_ms": 0.0, "device_ms": 0.0, "readback_ms": 0.0}
        starts = []
        # as many untimed warm-up steps as the main timing (the first of them
        # allocates the pinned result buffers)
        nw = max(1, args.warmup)
        for it in range(nw + args.e2e_steps):
            if it == nw:
                torch.cuda.synchronize()
                barrier(ws)
                t0 = time.perf_counter()
            ta = time.perf_counter()
            if it >= nw:
                starts.append(ta)
            one_step(ste, sub)
            tb = time.perf_counter()
            if it < nw:
                outs = ste.read_cube_sparse(out=outs) if sparse else ste.read_cube(device=False, out=outs)
            elif sparse:
                # the touched entries only (the same set every step): a
                # synchronous call, the last step's split into run and readback
                last = it == nw + args.e2e_steps - 1
                if last:
                    torch.cuda.current_stream().synchronize()
                tc = time.perf_counter()
                outs = ste.read_cube_sparse(out=outs)
                if last:
                    td = time.perf_counter()
                    split = {"queue_ms": (tb - ta) * 1e3, "device_ms": (tc - tb) * 1e3,
                             "readback_ms": (td - tc) * 1e3}
            elif it < nw + args.e2e_steps - 1:
                # every step reads its cube back; the copy overlaps the next step's
                ste.read_cube_async(outs)
            else:
                # the last step also splits its time: its run, then its readback
                torch.cuda.current_stream().synchronize()
                tc = time.perf_counter()
                ste.read_cube_async(outs)
                ste.wait_readback()
                td = time.perf_counter()
                split = {"queue_ms": (tb - ta) * 1e3, "device_ms": (tc - tb) * 1e3, "readback_ms": (td - tc) * 1e3}
        ste.wait_readback()
        t_end = time.perf_counter()
        dt = (t_end - t0) / args.e2e_steps
        # the arrays read back (and, sparse, the 8-byte count of touched entries)
        d2h = sum(v.numel() * v.element_size() for v in outs.values()) + (8 if sparse else 0)
        n_back = int(outs["index"].numel()) if sparse else int(outs["count"].numel())
        h2d = ste.h2d_bytes()   # what vista_run copied for the windows (the last step's; every step's is the same)
    finally:
        ste.close()
    dt = allmax(ws, dt)
    n_in = sum(1 for s in wl.spws if window_io(s, f0, df, wl.nrest)[0] > 0)
    return {"value": allsum(ws, n_vis) / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": dt * 1e3,
            "windows": "%d of the %d windows that reach the cube (%d visibilities, %.1f GB pinned on the host)" % (
                len(host), n_in, n_vis, pinned / 1e9),
            "link_gbs": (h2d + d2h) / dt / 1e9,
            "readback": ("the %d touched cube entries (index, sums and count: 28 B each)" % n_back if sparse
                         else "the whole cube (%d entries, 20 B each), overlapping the next step" % n_back),
            # host time between successive steps' starts (the host runs ahead
            # of the device by up to two steps, so single values are not a
            # step's device time; their spread shows this shared machine's noise)
            "step_starts_ms": [round((b - a) * 1e3, 1) for a, b in zip(starts, starts[1:] + [t_end])],
            "last_step_split": split}


def host_link_peak(nbytes=4 << 30, reps=3):
    """Pinned host <-> device copy rate: one large cudaMemcpyAsync each way,
    best of `reps`, timed by CUDA events on the current stream."""
    try:
        h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    except RuntimeError as exc:
        return {"error": str(exc)[:200]}
    h.fill_(1)
    stream = torch.cuda.current_stream()
    best = {}
    for name, dst, src in (("h2d_gbs", d, h), ("d2h_gbs", h, d)):
        t = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dst.copy_(src, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1) * 1e-3)
        best[name] = nbytes / min(t) / 1e9
    best["bytes"] = nbytes
    del h, d
    return best


def workload_name(wl):
    if wl.name == "batched":
        return ("batched: %d windows (%d sources), rows lognormal(median 20000, sigma_ln 1), 1-4 windows of "
                "128-3840 ch, 2/4 pol c64, aliased into a device pool; cube %dx%dx%dx%d" % (
                    len(wl.spws), len({s.source for s in wl.spws}), wl.nv, wl.nu, wl.nrest, wl.npol))
    s0 = wl.spws[0]
    storage = {torch.complex64: "c64", torch.float16: "FP16 pairs", torch.bfloat16: "BF16 pairs"}[s0.vis.dtype]
    extra = ""
    if wl.name.startswith("mixed"):
        extra = " (the sources of 64 whose windows reach the cube; lattice and cell size of all 64)"
    return "%s: %d windows (%d sources)%s, %d rows/window, %d ch x %d pol %s; cube %dx%dx%dx%d" % (
        wl.name, len(wl.spws), len({s.source for s in wl.spws}), extra, int(s0.vis.shape[0]),
        int(s0.vis.shape[1]), int(s0.vis.shape[2]), storage, wl.nv, wl.nu, wl.nrest, wl.npol)


def st_tuning_str(t):
    """The launch shape in effect (the library's defaults unless --tuning)."""
    return ", ".join("%s=%d" % kv for kv in t.items())


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    """The FP64 CPU oracle on the host cores, each step a bounded sample."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    nsample = max(1, args.ref_sample)
    from paper_2609_01897_gb300 import synth
    gen = {"alma_compact": synth.alma_compact, "mixed": synth.mixed, "wideband_hi": synth.wideband_hi}.get(args.config)
    if gen is not None:
        # geometry and channel axes of every source (the lattice and the cell
        # size depend on all), visibilities only for the sampled windows
        n = args.sources or {"wideband_hi": 24 if args.storage == "c64" else 48}.get(args.config, 64)
        meta = gen("cpu", n_sources=n, meta_only=True)
        f0, df = O.auto_lattice([s.freqs for s in meta.spws], [s.z for s in meta.spws], meta.nrest,
                                meta.central_freq)
        picked = windows_in_cube(meta, f0, df, nsample)
        ids = sorted({s.source for s in picked})
        wl = gen(dev, n_sources=n, src_ids=ids, du=meta.du)
        keep = {(s.source, float(s.freqs[0])) for s in picked}
        wl.spws = [s for s in wl.spws if (s.source, float(s.freqs[0])) in keep]
        if args.reproject:
            wl = synth.with_reprojection(wl, math.radians(-30.0))
        if args.storage != "c64":
            wl = synth.half_storage(wl, args.storage)
        spws = wl.spws
    else:
        wl = make_workload(argparse.Namespace(**vars(args)), 0, dev)
        f0, df = O.auto_lattice([s.freqs for s in wl.spws], [s.z for s in wl.spws], wl.nrest,
                                wl.central_freq)
        spws = windows_in_cube(wl, f0, df, nsample)
    srcs = [O.Source(s.uvw.cpu().numpy(), s.freqs, host_vis(s), s.weights.cpu().numpy(),
                     None if s.flags is None else s.flags.cpu().numpy(), s.l, s.m, s.z, s.pol_map,
                     radec=s.radec) for s in spws]
    cube = O.make_cube(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, f0, df, 0, 0)
    nthreads = os.cpu_count() or 1
    times, n = [], 0
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        out = O.stack(cube, srcs, nthreads=nthreads)
        dt = time.perf_counter() - t0
        n = int(out["stats"]["n_vis"])
        if it >= args.warmup:
            times.append(dt)
        del out
    ms = 1e3 * float(np.mean(times))
    value = n / (ms * 1e-3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(wl) + " (sample of %d windows per step)" % nsample,
                       "n_vis_per_step": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": "%d windows (%d visibilities) per step" % (nsample, n)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
