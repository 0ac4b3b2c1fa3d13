"""CUDA-graph replay of a run's device work: an unchanged source set is
replayed from a captured graph, the replay reads the arrays' current
contents, and any change of the set falls back to planning.  Results are
checked against the FP64 oracle like every other run."""
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


@pytest.fixture(scope="module")
def tiny():
    from paper_2609_01897_gb300 import synth
    return synth.tiny("cuda")


def _open(V, wl, precision):
    return V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, central_freq=wl.central_freq,
                   precision=precision)


def _add_all(st, spws):
    for s in spws:
        st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z, pol_map=s.pol_map)


def _cube(st):
    c = {k: v.cpu().numpy() for k, v in st.read_cube(f64=True).items()}
    c["sum_wv"] = c["sum_wv"][..., 0] + 1j * c["sum_wv"][..., 1]
    return c


def _scaled(orc, k):
    out = dict(orc)
    for key in ("sum_wv", "sum_w", "sum_wvv", "sum_wabs"):
        out[key] = orc[key] * k
    out["count"] = orc["count"] * k
    return out


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_replay_of_an_unchanged_set(V, tiny, prec):
    precision = V.PREC_MIXED if prec == "mixed" else V.PREC_FP64
    st = _open(V, tiny, precision)
    try:
        for _ in range(3):
            _add_all(st, tiny.spws)
            st.run()
        # run 1 plans, run 2 captures and launches the graph, run 3 replays it
        assert st.graph_runs() == 2
        g = _cube(st)
        stats = st.stats()
    finally:
        st.close()
    o = H.run_oracle(tiny)
    H.compare(g, _scaled(o, 3), H.TOL_MIXED if prec == "mixed" else H.TOL_FP64, what="3 runs, graph")
    assert stats["n_vis"] == 3 * int(o["stats"]["n_vis"])
    assert stats["n_stacked"] == 3 * int(o["stats"]["n_stacked"])


def test_replay_reads_current_contents(V, tiny):
    from paper_2609_01897_gb300 import synth
    spws = [synth.SourceSpw(s.uvw.clone(), s.freqs, s.vis.clone(), s.weights.clone(),
                      None if s.flags is None else s.flags.clone(), s.l, s.m, s.z, s.pol_map)
            for s in tiny.spws]
    st = _open(V, tiny, V.PREC_MIXED)
    try:
        for _ in range(2):
            _add_all(st, spws)
            st.run()
        assert st.graph_runs() == 1
        st.zero()
        # new contents in the same arrays: visibilities, weights and flags
        gen = torch.Generator(device="cuda").manual_seed(5)
        for s in spws:
            s.vis.copy_(torch.randn(s.vis.shape, dtype=s.vis.dtype, device="cuda", generator=gen))
            s.weights.mul_(0.5)
            if s.flags is not None:
                s.flags.copy_((torch.rand(s.flags.shape, device="cuda", generator=gen) < 0.2).to(s.flags.dtype))
        _add_all(st, spws)
        st.run()
        assert st.graph_runs() == 2
        g = _cube(st)
    finally:
        st.close()
    wl = synth.Workload("tiny-b", tiny.nu, tiny.nv, tiny.nrest, tiny.npol, tiny.du, tiny.dv, tiny.central_freq,
                        spws, rest_df=tiny.rest_df, rest_f0=tiny.rest_f0)
    H.compare(g, H.run_oracle(wl), H.TOL_MIXED, what="replay after new contents")


def test_changed_set_is_planned_again(V, tiny):
    st = _open(V, tiny, V.PREC_MIXED)
    try:
        for _ in range(2):
            _add_all(st, tiny.spws)
            st.run()
        assert st.graph_runs() == 1
        st.zero()
        _add_all(st, tiny.spws[:3])        # a different set: planned, not replayed
        st.run()
        assert st.graph_runs() == 1
        g = _cube(st)
        lat = st.lattice()
    finally:
        st.close()
    from paper_2609_01897_gb300 import synth
    wl = synth.Workload("tiny-3", tiny.nu, tiny.nv, tiny.nrest, tiny.npol, tiny.du, tiny.dv, tiny.central_freq,
                        tiny.spws[:3], rest_df=lat[1], rest_f0=lat[0])
    H.compare(g, H.run_oracle(wl), H.TOL_MIXED, what="changed set")


def test_graphs_can_be_disabled(V, tiny):
    st = _open(V, tiny, V.PREC_MIXED)
    try:
        st.enable_graphs(False)
        for _ in range(3):
            _add_all(st, tiny.spws)
            st.run()
        assert st.graph_runs() == 0
        cnt = st.read_cube(which=("count",))["count"].cpu().numpy()
    finally:
        st.close()
    o = H.run_oracle(tiny)
    assert np.array_equal(cnt.astype(np.int64), 3 * o["count"].astype(np.int64))
