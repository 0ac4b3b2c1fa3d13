"""Host-memory windows streamed through vista_run in waves (the read ->
compute pipeline): the copies of one wave run on the copy streams while the
wave before is stacked, two device staging slots taking turns, and the call
returns before the copies end.  Against the FP64 oracle: the tiny stack in
eight waves, a ragged stack (descending axes, pol maps) in at least four,
and the same cube as the device-memory path."""
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


def _host_run(V, wl, wave_bytes, runs=1):
    st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, rest_f0=wl.rest_f0, rest_df=wl.rest_df,
                 central_freq=wl.central_freq)
    try:
        st.set_wave_bytes(wave_bytes)
        host = []
        for s in wl.spws:
            host.append([a.cpu().pin_memory() if isinstance(a, torch.Tensor) else a
                         for a in (s.uvw, s.vis, s.weights, s.flags)])
        for _ in range(runs):
            for s, (u, v, w, f) in zip(wl.spws, host):
                st.add_source(u, s.freqs, v, w, f, l=s.l, m=s.m, z=s.z, pol_map=s.pol_map)
            st.run()
        waves = st.waves()
        cube = st.read_cube(device=True, f64=True)
        out = {k: v.cpu().numpy() for k, v in cube.items()}
        out["sum_wv"] = out["sum_wv"][..., 0] + 1j * out["sum_wv"][..., 1]
        out["stats"] = st.stats()
        return out, waves
    finally:
        st.close()


def test_tiny_in_eight_waves(V):
    from paper_2609_01897_gb300 import synth
    wl = synth.tiny("cuda")
    g, waves = _host_run(V, wl, 1 << 20)      # about one window per wave
    assert waves >= 4, waves
    o = H.run_oracle(wl)
    H.compare(g, o, H.TOL_MIXED, what="tiny, streamed")
    H.stats_equal(g, o)


def test_ragged_in_waves_and_repeated_runs(V):
    from paper_2609_01897_gb300 import synth
    wl = synth.random_case(23, "cuda", nsrc=6, max_rows=400, descending=True, with_pol_map=True)
    g, waves = _host_run(V, wl, 64 << 10, runs=2)
    assert waves >= 4, waves
    o = H.run_oracle(wl)
    o2 = {"sum_wv": 2 * o["sum_wv"], "sum_w": 2 * o["sum_w"], "sum_wvv": 2 * o["sum_wvv"],
          "sum_wabs": 2 * o["sum_wabs"], "count": 2 * o["count"]}
    H.compare(g, o2, H.TOL_MIXED, what="ragged, streamed twice")


def test_streamed_equals_device_path(V):
    from paper_2609_01897_gb300 import synth
    wl = synth.tiny("cuda")
    g, _ = _host_run(V, wl, 2 << 20)
    d = H.run_gpu(wl)
    np.testing.assert_array_equal(g["count"], d["count"])
    np.testing.assert_allclose(g["sum_w"], d["sum_w"], rtol=1e-6, atol=1e-6)


def test_async_readback_overlaps_runs_and_matches(V):
    """vista_read_cube_async after each streamed run (the next run's copies
    overlap the previous readback): every readback equals the cube after its
    run, read synchronously, and the oracle's sums times the run count."""
    from paper_2609_01897_gb300 import synth
    wl = synth.tiny("cuda")
    st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, rest_f0=wl.rest_f0, rest_df=wl.rest_df,
                 central_freq=wl.central_freq)
    try:
        st.set_wave_bytes(1 << 20)
        host = [[a.cpu().pin_memory() if isinstance(a, torch.Tensor) else a
                 for a in (s.uvw, s.vis, s.weights, s.flags)] for s in wl.spws]
        outs = [st.read_cube(device=False) for _ in range(3)]   # pinned buffers (a zero cube)
        for r in range(3):
            for s, (u, v, w, f) in zip(wl.spws, host):
                st.add_source(u, s.freqs, v, w, f, l=s.l, m=s.m, z=s.z, pol_map=s.pol_map)
            st.run()
            st.read_cube_async(outs[r])          # returns at once; the next run is queued behind it
        st.wait_readback()
        final = st.read_cube(device=False)
        assert st.h2d_bytes() > 0
    finally:
        st.close()
    o = H.run_oracle(wl)
    for r in range(3):
        g = {k: v.numpy().astype(np.float64) for k, v in outs[r].items()}
        g["sum_wv"] = g["sum_wv"][..., 0] + 1j * g["sum_wv"][..., 1]
        g["count"] = outs[r]["count"].numpy().astype(np.uint64)
        k = r + 1
        ok = {"sum_wv": k * o["sum_wv"], "sum_w": k * o["sum_w"], "sum_wvv": k * o["sum_wvv"],
              "sum_wabs": k * o["sum_wabs"], "count": k * o["count"]}
        H.compare(g, ok, H.TOL_MIXED, what="async readback after run %d" % k)
    for key in ("count", "sum_w"):
        assert torch.equal(outs[2][key], final[key]), key


@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_streamed_half_storage(V, kind):
    """Host windows in 16-bit storage (per-window power-of-two scales)
    streamed in several waves, against the oracle on the stored values."""
    from paper_2609_01897_gb300 import synth
    wl = synth.tiny("cuda")
    st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, rest_f0=wl.rest_f0, rest_df=wl.rest_df,
                 central_freq=wl.central_freq)
    deq = {}
    try:
        st.set_wave_bytes(256 << 10)
        for s in wl.spws:
            q, scale, d = H.quantise(s.vis, kind)
            deq[id(s)] = d
            st.add_source(s.uvw.cpu().pin_memory(), s.freqs, q.cpu().pin_memory(), s.weights.cpu().pin_memory(),
                          s.flags.cpu().pin_memory(), l=s.l, m=s.m, z=s.z, vis_scale=scale)
        st.run()
        waves = st.waves()
        cube = st.read_cube(device=True, f64=True)
        g = {k: v.cpu().numpy() for k, v in cube.items()}
    finally:
        st.close()
    assert waves >= 4, waves
    g["sum_wv"] = g["sum_wv"][..., 0] + 1j * g["sum_wv"][..., 1]
    o = H.run_oracle(wl, dequant=deq)
    H.compare(g, o, H.TOL_MIXED, what="streamed %s" % kind)
