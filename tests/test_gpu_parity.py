"""GPU parity: libvista (through its C ABI) against the FP64 CPU oracle on the
same seeded inputs.  Bins and counts exact, sums within the stated tolerance,
phasors within 1e-5 rad (mixed) / 1e-9 rad (FP64)."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from tests import gpu_helpers as H  # noqa: E402

ARCSEC = math.pi / 180 / 3600


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_01897_gb300 import build
    build.build()
    from paper_2609_01897_gb300 import vista
    vista.lib()
    return vista


@pytest.fixture(scope="module")
def tiny():
    from paper_2609_01897_gb300 import synth
    return synth.tiny("cuda")


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("mode", [0, 1])
def test_tiny(V, tiny, prec, mode):
    p = V.PREC_MIXED if prec == "mixed" else V.PREC_FP64
    g = H.run_gpu(tiny, precision=p, bin_mode=mode)
    o = H.run_oracle(tiny, bin_mode=mode)
    assert g["lattice"] == o["lattice"]
    H.compare(g, o, H.TOL_MIXED if prec == "mixed" else H.TOL_FP64, what="tiny " + prec)
    H.stats_equal(g, o)
    assert o["stats"]["n_stacked"] > 0.9 * o["stats"]["n_vis"]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_ragged_cases(V, seed, prec):
    """Ragged rows (zero included), odd channel counts, 1/2/4 pols, descending
    axes, pol maps, off-grid rows and out-of-lattice channels."""
    from paper_2609_01897_gb300 import synth
    wl = synth.random_case(100 + seed, "cuda", nsrc=4, descending=seed % 2 == 1,
                           with_pol_map=seed % 3 == 2)
    p = V.PREC_MIXED if prec == "mixed" else V.PREC_FP64
    mode = seed % 2
    fold = seed % 3 == 1
    tuning = [None, dict(rows_per_item=7, chans_per_lane=1), dict(rows_per_item=3, chans_per_lane=2, sort_rows=0),
              dict(rows_per_item=256, chans_per_lane=4, warps_per_cta=8)][seed % 4]
    g = H.run_gpu(wl, precision=p, bin_mode=mode, fold=fold, tuning=tuning)
    o = H.run_oracle(wl, bin_mode=mode, fold=fold)
    H.compare(g, o, H.TOL_MIXED if prec == "mixed" else H.TOL_FP64, what="random %d" % seed)
    H.stats_equal(g, o)
    assert o["stats"]["n_dropped_uv"] > 0


def _long_baseline_case(seed, nrow=300, nchan=960, offset=60 * ARCSEC):
    """Mixed-workload geometry: baselines to 16 km, 960 channels at 340 GHz,
    offsets up to 60" (|tau nu / c| reaches thousands of turns)."""
    from paper_2609_01897_gb300 import synth
    rng = np.random.default_rng(seed)
    enu = synth.array_enu(43, 8000.0, rng)
    uvw = synth.uvw_tracks(enu, -23.0, -30.0, 3, 30.0, 0.4)[:nrow]
    f = 340e9 + 1.953125e6 * np.arange(nchan)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    vis = torch.complex(torch.randn((nrow, nchan, 2), generator=g, device="cuda"),
                        torch.randn((nrow, nchan, 2), generator=g, device="cuda")).to(torch.complex64)
    spw = synth.SourceSpw(torch.as_tensor(uvw, device="cuda"), f, vis,
                          torch.ones((nrow, 2), dtype=torch.float32, device="cuda"), None,
                          offset, -0.8 * offset, 2.5)
    n = 256
    du = 2 * 1.0001 * np.abs(uvw[:, :2]).max() * f.max() / H.C_LIGHT / n
    return synth.Workload("longbl", n, n, 1024, 2, du, du, 0.0, [spw])


@pytest.mark.parametrize("cpl", [1, 2, 4])
def test_phasor_and_cells_mixed(V, cpl):
    wl = _long_baseline_case(7)
    wl.central_freq = 340e9 * 3.5 + 0.5 * 960 * 1.953125e6 * 3.5
    s = wl.spws[0]
    st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, central_freq=wl.central_freq)
    st.set_tuning(chans_per_lane=cpl)
    st.add_source(s.uvw, s.freqs, s.vis, s.weights, None, l=s.l, m=s.m, z=s.z)
    st.run()
    nrow, nchan = s.vis.shape[0], s.vis.shape[1]
    ph = st.debug_phasors(0, nrow, nchan).cpu().numpy()
    cl = st.debug_cells(0, nrow, nchan).cpu().numpy()
    st.close()
    osrc = H.oracle_sources(wl)[0]
    from oracle import oracle as O
    pho = O.phasors(osrc)
    f0, df = H.lattice_of(wl)
    clo = O.cells(O.make_cube(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, f0, df, 0, 0), osrc)
    read = cl[..., 0] != -7
    assert read.mean() > 0.5
    pg = ph[..., 0] + 1j * ph[..., 1]
    err = H.phase_error(pg[read], pho[read])
    assert err <= H.PHASE_TOL_MIXED, err
    np.testing.assert_array_equal(cl[read], clo[read])
    # the case reaches large unreduced phases: max |tau nu_k / c| over the
    # rows and channels read, from the inputs (not the reduced angle)
    u = s.uvw.cpu().numpy()
    tau = u[:, 0] * s.l + u[:, 1] * s.m + u[:, 2] * (np.sqrt(1 - s.l ** 2 - s.m ** 2) - 1)
    turns = np.abs(tau[:, None] * s.freqs[None, :] / H.C_LIGHT)[read].max()
    assert turns > 1e3, turns


def test_phasor_and_cells_fp64(V):
    wl = _long_baseline_case(8, nrow=120)
    wl.central_freq = 340e9 * 3.5 + 0.5 * 960 * 1.953125e6 * 3.5
    s = wl.spws[0]
    st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, central_freq=wl.central_freq,
                 precision=V.PREC_FP64)
    st.add_source(s.uvw, s.freqs, s.vis, s.weights, None, l=s.l, m=s.m, z=s.z)
    st.run()
    nrow, nchan = s.vis.shape[0], s.vis.shape[1]
    ph = st.debug_phasors(0, nrow, nchan).cpu().numpy()
    cl = st.debug_cells(0, nrow, nchan).cpu().numpy()
    st.close()
    from oracle import oracle as O
    osrc = H.oracle_sources(wl)[0]
    f0, df = H.lattice_of(wl)
    clo = O.cells(O.make_cube(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, f0, df, 0, 0), osrc)
    read = cl[..., 0] != -7
    assert read.mean() > 0.5
    pg = ph[..., 0] + 1j * ph[..., 1]
    assert H.phase_error(pg[read], O.phasors(osrc)[read]) <= H.PHASE_TOL_FP64
    np.testing.assert_array_equal(cl[read], clo[read])


def test_cells_at_exact_boundaries(V):
    """Rows whose u*s_k lands on (or one ulp beside) an integer cell edge:
    the guarded FP32 path must fall back to the FP64 product and agree with
    the oracle bit for bit."""
    from paper_2609_01897_gb300 import synth
    nchan = 64
    f = 100e9 + 15.625e6 * np.arange(nchan)
    du = 1000.0
    gu = 1.0 / (H.C_LIGHT * du)
    rows = []
    rng = np.random.default_rng(3)
    for i in range(256):
        k = int(rng.integers(0, nchan))
        n = int(rng.integers(-60, 60))
        s_k = f[k] * gu
        u = n / s_k
        u = np.nextafter(u, u + (i % 3 - 1)) if i % 3 != 1 else u
        v = (int(rng.integers(-60, 60)) + 0.5) / s_k
        rows.append([u, v, 0.0])
    uvw = np.array(rows)
    vis = torch.ones((256, nchan, 1), dtype=torch.complex64, device="cuda")
    spw = synth.SourceSpw(torch.as_tensor(uvw, device="cuda"), f, vis,
                          torch.ones((256, 1), dtype=torch.float32, device="cuda"), None, 0.0, 0.0, 0.0)
    wl = synth.Workload("edges", 128, 128, 8, 1, du, du, 0.0, [spw], rest_df=0.2e9, rest_f0=99.9e9)
    for prec in (V.PREC_MIXED, V.PREC_FP64):
        st = V.Stack(wl.nu, wl.nv, wl.nrest, 1, du, du, rest_f0=wl.rest_f0, rest_df=wl.rest_df,
                     precision=prec)
        st.add_source(spw.uvw, f, vis, spw.weights, None, l=0.0, m=0.0, z=0.0)
        st.run()
        cl = st.debug_cells(0, 256, nchan).cpu().numpy()
        st.close()
        from oracle import oracle as O
        f0, df = H.lattice_of(wl)
        clo = O.cells(O.make_cube(128, 128, 8, 1, du, du, f0, df, 0, 0), H.oracle_sources(wl)[0])
        read = cl[..., 0] != -7
        assert read.mean() > 0.9
        np.testing.assert_array_equal(cl[read], clo[read])


@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_half_storage(V, tiny, kind):
    qs, scales, deq = [], [], {}
    for s in tiny.spws:
        q, sc, d = H.quantise(s.vis, kind)
        qs.append(q)
        scales.append(sc)
        deq[id(s)] = d
    g = H.run_gpu(tiny, vis_override=qs, scales=scales)
    o = H.run_oracle(tiny, dequant=deq)
    H.compare(g, o, H.TOL_MIXED, what="tiny " + kind)
    H.stats_equal(g, o)


def test_host_memory_mode_matches_device(V, tiny):
    a = H.run_gpu(tiny)
    b = H.run_gpu(tiny, host_mem=True)
    np.testing.assert_array_equal(a["count"], b["count"])
    o = H.run_oracle(tiny)
    H.compare(b, o, H.TOL_MIXED, what="host-mem")
    for k in ("n_vis", "n_flagged", "n_dropped_uv", "n_stacked"):
        assert a["stats"][k] == b["stats"][k]


def test_runs_are_additive(V, tiny):
    from paper_2609_01897_gb300 import synth
    st = V.Stack(tiny.nu, tiny.nv, tiny.nrest, tiny.npol, tiny.du, tiny.dv, central_freq=tiny.central_freq)
    half = len(tiny.spws) // 2
    for part in (tiny.spws[:half], tiny.spws[half:]):
        for s in part:
            st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z)
        st.run()
    cube = st.read_cube(f64=True)
    stats = st.stats()
    st.close()
    # the lattice was fixed by the first half: the oracle uses the same one
    f0, df = H.O.auto_lattice([s.freqs for s in tiny.spws[:half]], [s.z for s in tiny.spws[:half]],
                              tiny.nrest, tiny.central_freq)
    wl = synth.Workload("tiny", tiny.nu, tiny.nv, tiny.nrest, tiny.npol, tiny.du, tiny.dv,
                        tiny.central_freq, tiny.spws, rest_df=df, rest_f0=f0)
    o = H.run_oracle(wl)
    g = {k: v.cpu().numpy() for k, v in cube.items()}
    g["sum_wv"] = g["sum_wv"][..., 0] + 1j * g["sum_wv"][..., 1]
    H.compare(g, o, H.TOL_MIXED, what="additive")
    assert stats["n_stacked"] == o["stats"]["n_stacked"]


def test_zero_cube_and_rerun(V, tiny):
    st = V.Stack(tiny.nu, tiny.nv, tiny.nrest, tiny.npol, tiny.du, tiny.dv, central_freq=tiny.central_freq)
    s = tiny.spws[0]
    for _ in range(2):
        st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z)
        st.run()
    c2 = st.read_cube(which=("count",))["count"].clone()
    st.zero()
    assert int(st.read_cube(which=("count",))["count"].sum()) == 0
    assert st.stats()["n_vis"] == 0
    st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z)
    st.run()
    c1 = st.read_cube(which=("count",))["count"]
    st.close()
    assert torch.equal(c2, 2 * c1)


def test_errors(V, tiny):
    s = tiny.spws[0]
    st = V.Stack(tiny.nu, tiny.nv, tiny.nrest, tiny.npol, tiny.du, tiny.dv, central_freq=tiny.central_freq)
    with pytest.raises(V.VistaError) as e:
        st.run()
    assert e.value.code == V.E_STATE
    with pytest.raises(V.VistaError) as e:
        st.lattice()
    assert e.value.code == V.E_STATE
    bad = [dict(l=0.8, m=0.7), dict(z=-1.0), dict(z=float("nan"))]
    for b in bad:
        kw = dict(l=s.l, m=s.m, z=s.z)
        kw.update(b)
        with pytest.raises(V.VistaError) as e:
            st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, **kw)
        assert e.value.code == V.E_ARG
    f = s.freqs.copy()
    f[3] = f[2]
    with pytest.raises(V.VistaError) as e:
        st.add_source(s.uvw, f, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z)
    assert e.value.code == V.E_ARG
    raw =torch.empty(s.vis.numel() + 1, dtype=torch.complex64, device="cuda")[1:].view(s.vis.shape)
    with pytest.raises(V.VistaError) as e:
        st.add_source(s.uvw, s.freqs, raw, s.weights, s.flags, l=s.l, m=s.m, z=s.z)
    assert e.value.code == V.E_ARG
    with pytest.raises(V.VistaError) as e:
        st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z, pol_map=[0, 5])
    assert e.value.code == V.E_ARG
    # a failed add leaves nothing queued
    with pytest.raises(V.VistaError):
        st.run()
    st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z)
    st.run()
    assert st.stats()["n_vis"] > 0
    h = st.h
    st.close()
    assert V.lib().vista_run(h) == V.E_STATE
    assert V.lib().vista_add_source(h, None) == V.E_STATE


def test_failed_allocation_leaves_no_pending_error(V, tiny):
    # a cube of 1024 x 1024 cells x 262144 rest channels x 4 pols needs
    # about 57 TB: cudaMalloc refuses it at once and the open reports
    # VISTA_E_NOMEM.  The refused allocation must not stay behind as the
    # thread's last CUDA error, where the next launch check (torch's own, or
    # the library's in a later run) would take it for its own failure.
    with pytest.raises(V.VistaError) as e:
        V.Stack(1024, 1024, 262144, 4, tiny.du, tiny.dv, central_freq=tiny.central_freq)
    assert e.value.code == V.E_NOMEM
    x = torch.arange(1024, dtype=torch.float32, device="cuda") * 2.0
    torch.cuda.synchronize()
    assert float(x.sum()) == 1023.0 * 1024.0
    g = H.run_gpu(tiny)
    o = H.run_oracle(tiny)
    H.compare(g, o, H.TOL_MIXED, what="tiny after a refused allocation")


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_sparse_readback_matches_dense(V, tiny, prec):
    """vista_read_cube_sparse: the entries with count > 0, in entry order, with
    the values vista_read_cube gives (bit for bit), into host and device
    arrays; the entries with count 0 hold zero sums; cap = 0 only counts, a
    smaller cap returns E_RANGE with the count, bad arguments E_ARG; a zeroed
    cube has no touched entry."""
    import ctypes as C
    p = V.PREC_MIXED if prec == "mixed" else V.PREC_FP64
    st = V.Stack(tiny.nu, tiny.nv, tiny.nrest, tiny.npol, tiny.du, tiny.dv, central_freq=tiny.central_freq,
                 precision=p)
    try:
        for s in tiny.spws:
            st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z)
        st.run()
        dense = st.read_cube(device=True)
        cnt = dense["count"].reshape(-1)
        want = torch.nonzero(cnt != 0).reshape(-1)
        assert 0 < want.numel() < cnt.numel()
        flat = {"sum_wv": dense["sum_wv"].reshape(-1, 2), "sum_w": dense["sum_w"].reshape(-1),
                "sum_wvv": dense["sum_wvv"].reshape(-1), "count": cnt}
        for k in ("sum_wv", "sum_w", "sum_wvv"):
            assert (flat[k][cnt == 0] == 0).all(), k
        out = None
        for device in (False, True, False):
            sp = st.read_cube_sparse(device=device, out=out)
            assert sp["index"].is_cuda == device
            assert torch.equal(sp["index"].cuda(), want)
            for k in ("sum_wv", "sum_w", "sum_wvv", "count"):
                assert torch.equal(sp[k].cuda(), flat[k][want]), k
            out = sp if not device else None
        L, n = V.lib(), C.c_int64(-1)
        assert L.vista_read_cube_sparse(st.h, 0, None, None, None, None, None, C.byref(n), 0) == V.VISTA_OK
        assert n.value == want.numel()
        small = torch.empty(5, dtype=torch.int64, pin_memory=True)
        n.value = -1
        assert L.vista_read_cube_sparse(st.h, 5, small.data_ptr(), None, None, None, None, C.byref(n), 0) == V.E_RANGE
        assert n.value == want.numel() and "touched" in V.last_error(st.h)
        assert L.vista_read_cube_sparse(st.h, -1, None, None, None, None, None, C.byref(n), 0) == V.E_ARG
        assert L.vista_read_cube_sparse(st.h, 5, None, None, None, None, None, C.byref(n), 0) == V.E_ARG
        assert L.vista_read_cube_sparse(st.h, 5, small.data_ptr(), None, None, None, None, None, 0) == V.E_ARG
        st.zero()
        assert st.read_cube_sparse()["index"].numel() == 0
    finally:
        st.close()


def test_all_flagged_and_empty(V, tiny):
    s = tiny.spws[0]
    st = V.Stack(tiny.nu, tiny.nv, tiny.nrest, tiny.npol, tiny.du, tiny.dv, central_freq=tiny.central_freq)
    st.add_source(s.uvw, s.freqs, s.vis, s.weights, torch.ones_like(s.flags), l=s.l, m=s.m, z=s.z)
    st.add_source(s.uvw[:0], s.freqs, s.vis[:0], s.weights[:0], s.flags[:0], l=s.l, m=s.m, z=s.z)
    st.run()
    c = st.read_cube()
    stats = st.stats()
    st.close()
    assert int(c["count"].sum()) == 0 and float(c["sum_w"].abs().sum()) == 0.0
    assert stats["n_flagged"] == stats["n_vis"] > 0 and stats["n_stacked"] == 0


def test_host_readback_into_caller_buffers(V, tiny):
    st = V.Stack(tiny.nu, tiny.nv, tiny.nrest, tiny.npol, tiny.du, tiny.dv, central_freq=tiny.central_freq)
    try:
        for s in tiny.spws:
            st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z)
        st.run()
        dev = {k: v.cpu() for k, v in st.read_cube(device=True).items()}
        host = st.read_cube(device=False)
        ptrs = {k: v.data_ptr() for k, v in host.items()}
        for v in host.values():
            v.zero_()
        again = st.read_cube(device=False, out=host)
        with pytest.raises(ValueError):
            st.read_cube(device=False, out={"sum_w": host["sum_w"][:1]}, which=("sum_w",))
    finally:
        st.close()
    for k in dev:
        assert again[k].data_ptr() == ptrs[k]          # filled in place
        assert torch.equal(again[k], dev[k]), k
