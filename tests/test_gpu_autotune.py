"""The launch-shape autotuner: it returns a valid shape, keeps it, leaves the
queue in place and the cube zero, and the run that follows matches the FP64
oracle."""
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


def test_autotune_then_run(V):
    from paper_2609_01897_gb300 import synth
    wl = synth.tiny("cuda")
    st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, central_freq=wl.central_freq)
    try:
        for s in wl.spws:
            st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z, pol_map=s.pol_map)
        best = st.autotune(budget=5, reps=1)
        assert best["rows_per_item"] in (32, 48, 64, 96)
        assert best["chans_per_lane"] in (1, 2)
        assert best["warps_per_cta"] in (2, 4, 8)
        assert best["prefetch_rows"] in (2, 4, 8)
        assert st.tuning() == best
        assert int(st.read_cube(which=("count",))["count"].sum()) == 0
        assert st.stats()["n_vis"] == 0
        st.run()                       # the queue autotune left in place
        g = {k: v.cpu().numpy() for k, v in st.read_cube(f64=True).items()}
        g["sum_wv"] = g["sum_wv"][..., 0] + 1j * g["sum_wv"][..., 1]
        stats = st.stats()
    finally:
        st.close()
    o = H.run_oracle(wl)
    H.compare(g, o, H.TOL_MIXED, what="after autotune")
    assert int(stats["n_stacked"]) == int(o["stats"]["n_stacked"])


def test_autotune_needs_a_queue(V):
    from paper_2609_01897_gb300 import synth
    wl = synth.tiny("cuda")
    st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, central_freq=wl.central_freq)
    try:
        with pytest.raises(RuntimeError):
            st.autotune()
    finally:
        st.close()
