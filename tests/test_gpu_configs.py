"""The precision and wideband configurations, in the shapes of their full
workloads:

* mixed precision (4 windows x 960 channels at 340-356 GHz, baselines up to
  16 km, offsets up to 60", |tau nu / c| up to ~5e3 turns): every source of
  the 64 whose windows reach the cube (the cube's lattice and cell size are
  those of all 64), stored as complex64, FP16 and BF16 with per-window
  scales.  Each run is compared with the FP64 oracle on the inputs it stacked
  (dequantised for the 16-bit storage: the 1e-5 bar) and, for the 16-bit
  storage, also with the oracle on the complex64 originals (the storage
  error, stated, not bounded).  The worst error of every output is printed.
* wideband HI (4096 channels over 856-1712 MHz, cube 512 x 512 x 2048 x 2):
  8 of the 24 sources (lattice and cell size of all 24), the mixed path
  against the plain FP64 GPU path on every cube entry, and the FP64 oracle
  on sampled planes; and the same for the complex-half variant (48 sources
  stored as FP16 pairs)."""
import json

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from tests import gpu_helpers as H  # noqa: E402


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_01897_gb300 import build
    build.build()
    from paper_2609_01897_gb300 import vista
    vista.lib()
    return vista


def _lattice_and_ids(meta, V):
    f0, df = H.O.auto_lattice([s.freqs for s in meta.spws], [s.z for s in meta.spws], meta.nrest,
                              meta.central_freq)
    ids = set()
    for s in meta.spws:
        _, nb, _ = V.plan_channels(s.freqs, s.z, f0, df, meta.nrest, V.BIN_OVERLAP)
        if (nb > 0).any():
            ids.add(s.source)
    return f0, df, sorted(ids)


def test_mixed_precision_config(V):
    from paper_2609_01897_gb300 import synth
    meta = synth.mixed("cpu", meta_only=True)
    f0, df, ids = _lattice_and_ids(meta, V)
    assert ids
    wl = synth.mixed("cuda", src_ids=ids, du=meta.du)
    wl.rest_f0, wl.rest_df = f0, df
    o64 = H.run_oracle(wl, nthreads=16)
    assert o64["count"].sum() > 1e8
    report = {}
    g = H.run_gpu(wl)
    report["complex64"] = H.compare(g, o64, H.TOL_MIXED, what="mixed config c64")
    for kind in ("f16", "bf16"):
        q, scales, deq = [], [], {}
        for s in wl.spws:
            t, sc, d = H.quantise(s.vis, kind)
            q.append(t)
            scales.append(sc)
            deq[id(s)] = d
        gq = H.run_gpu(wl, vis_override=q, scales=scales)
        oq = H.run_oracle(wl, dequant=deq, nthreads=16)
        report[kind] = H.compare(gq, oq, H.TOL_MIXED, what="mixed config " + kind)
        # storage error against the complex64 originals: stated, not bounded
        report[kind + " vs complex64 inputs"] = {
            "sum_wv": float(np.max(np.abs(gq["sum_wv"] - o64["sum_wv"]) / np.maximum(o64["sum_wabs"], 1e-300))),
            "sum_w": float(np.max(np.abs(gq["sum_w"] - o64["sum_w"]) / np.maximum(o64["sum_w"], 1e-300))),
            "sum_wvv": float(np.max(np.abs(gq["sum_wvv"] - o64["sum_wvv"]) / np.maximum(o64["sum_wvv"], 1e-300))),
        }
    print("mixed-precision config, worst error per output:", json.dumps(report))


def test_wideband_hi(V):
    from paper_2609_01897_gb300 import synth
    meta = synth.wideband_hi("cpu", meta_only=True)
    f0, df, _ = _lattice_and_ids(meta, V)
    wl = synth.wideband_hi("cuda", src_ids=range(8), du=meta.du)
    cubes, stats = {}, {}
    for prec in (V.PREC_MIXED, V.PREC_FP64):
        st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, rest_f0=f0, rest_df=df, precision=prec)
        try:
            for s in wl.spws:
                st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z)
            st.run()
            cubes[prec] = st.read_cube(device=True, f64=True)
            stats[prec] = st.stats()
        finally:
            st.close()
    m, d = cubes[V.PREC_MIXED], cubes[V.PREC_FP64]
    assert torch.equal(m["count"], d["count"])
    assert int(d["count"].sum()) > 1e9
    for key in ("sum_w", "sum_wvv"):
        err = (m[key] - d[key]).abs()
        assert bool((err <= H.TOL_MIXED * d[key].abs() + 1e-300).all()), key
    scale = torch.sqrt(d["sum_w"] * d["sum_wvv"])
    err = (m["sum_wv"] - d["sum_wv"]).abs().amax(dim=-1)
    assert bool((err <= H.TOL_MIXED * scale + 1e-300).all()), "sum_wv"
    for k in ("n_vis", "n_flagged", "n_dropped_uv", "n_stacked"):
        assert int(stats[V.PREC_MIXED][k]) == int(stats[V.PREC_FP64][k]), k

    # the FP64 oracle on two sampled planes, for the first two sources
    planes = [200, 300]
    sel = torch.tensor(planes, device="cuda")
    del cubes, m, d, scale, err
    torch.cuda.empty_cache()
    sub = synth.wideband_hi("cuda", src_ids=range(2), du=meta.du)
    st = V.Stack(sub.nu, sub.nv, sub.nrest, sub.npol, sub.du, sub.dv, rest_f0=f0, rest_df=df)
    try:
        for s in sub.spws:
            st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z)
        st.run()
        c = st.read_cube(device=True, f64=True)
        g = {k: v.index_select(0, sel).cpu().numpy() for k, v in c.items()}
        g["sum_wv"] = g["sum_wv"][..., 0] + 1j * g["sum_wv"][..., 1]
        del c
    finally:
        st.close()
    sub.rest_f0, sub.rest_df = f0, df
    o = H.run_oracle(sub, iv_select=planes, nthreads=16)
    assert o["count"].sum() > 1e5
    errs = H.compare(g, o, H.TOL_MIXED, what="wideband HI sampled planes")
    print("wideband HI, sampled planes, worst errors:", json.dumps(errs))


def test_wideband_hi_half_storage(V):
    """The complex-half wideband stack (48 sources stored as FP16 pairs): 8 of
    its sources on the lattice and cell size of all 48, the mixed path
    against the plain FP64 GPU path reading the same stored values on every
    cube entry, and the FP64 oracle on the dequantised values on a sampled
    plane."""
    from paper_2609_01897_gb300 import synth
    meta = synth.wideband_hi("cpu", n_sources=48, meta_only=True)
    f0, df, _ = _lattice_and_ids(meta, V)
    wl = synth.wideband_hi("cuda", n_sources=48, src_ids=range(8), du=meta.du, storage="f16")
    assert all(s.vis.dtype == torch.float16 for s in wl.spws)
    cubes, stats = {}, {}
    for prec in (V.PREC_MIXED, V.PREC_FP64):
        st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, rest_f0=f0, rest_df=df, precision=prec)
        try:
            for s in wl.spws:
                st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z,
                              vis_scale=s.vis_scale)
            st.run()
            cubes[prec] = st.read_cube(device=True, f64=True)
            stats[prec] = st.stats()
        finally:
            st.close()
    m, d = cubes[V.PREC_MIXED], cubes[V.PREC_FP64]
    assert torch.equal(m["count"], d["count"])
    assert int(d["count"].sum()) > 1e9
    worst = {}
    for key in ("sum_w", "sum_wvv"):
        err = (m[key] - d[key]).abs()
        assert bool((err <= H.TOL_MIXED * d[key].abs() + 1e-300).all()), key
        worst[key] = float((err / d[key].abs().clamp_min(1e-300)).max())
    scale = torch.sqrt(d["sum_w"] * d["sum_wvv"])
    err = (m["sum_wv"] - d["sum_wv"]).abs().amax(dim=-1)
    assert bool((err <= H.TOL_MIXED * scale + 1e-300).all()), "sum_wv"
    worst["sum_wv"] = float((err / scale.clamp_min(1e-300)).max())
    for k in ("n_vis", "n_flagged", "n_dropped_uv", "n_stacked"):
        assert int(stats[V.PREC_MIXED][k]) == int(stats[V.PREC_FP64][k]), k
    print("wideband HI, FP16 storage, mixed vs FP64 GPU path, worst errors:", json.dumps(worst))

    # the oracle on the dequantised values of the first source, one plane
    plane = 256
    sel = torch.tensor([plane], device="cuda")
    del cubes, m, d, scale, err
    torch.cuda.empty_cache()
    sub = synth.Workload("hi-f16-1", wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, wl.central_freq,
                         wl.spws[:1], rest_df=df, rest_f0=f0)
    st = V.Stack(sub.nu, sub.nv, sub.nrest, sub.npol, sub.du, sub.dv, rest_f0=f0, rest_df=df)
    try:
        s = sub.spws[0]
        st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z, vis_scale=s.vis_scale)
        st.run()
        c = st.read_cube(device=True, f64=True)
        g = {k: v.index_select(0, sel).cpu().numpy() for k, v in c.items()}
        g["sum_wv"] = g["sum_wv"][..., 0] + 1j * g["sum_wv"][..., 1]
        del c
    finally:
        st.close()
    s = sub.spws[0]
    deq = {id(s): torch.view_as_complex(s.vis.to(torch.float64).mul_(s.vis_scale)).cpu().numpy()}
    o = H.run_oracle(sub, iv_select=[plane], dequant=deq, nthreads=16)
    assert o["count"].sum() > 1e4
    errs = H.compare(g, o, H.TOL_MIXED, what="wideband HI FP16, sampled plane")
    print("wideband HI, FP16 storage, sampled plane vs the oracle:", json.dumps(errs))
