"""The paper's per-row output (Eq. 3, vista_regrid_rows) against the oracle's
plain per-row products: every row of every tiny window, both binning modes,
16-bit storage, the rest-frame uvw, and the state error before the lattice
is fixed."""
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


def _check(g_vis, g_w, o_vis, o_w, vis_scale):
    g_vis, g_w = g_vis.cpu().numpy().astype(np.complex128), g_w.cpu().numpy().astype(np.float64)
    # FP64 on both sides, rounded once to FP32 on output
    np.testing.assert_allclose(g_w, o_w, rtol=1e-6, atol=1e-7)
    err = np.abs(g_vis - o_vis)
    assert (err <= 1e-6 * (np.abs(o_vis) + vis_scale)).all(), float(err.max())
    assert (o_w > 0).sum() > 0


@pytest.mark.parametrize("mode", ["overlap", "nearest"])
def test_regrid_rows_against_oracle(V, tiny, mode):
    bin_mode = V.BIN_OVERLAP if mode == "overlap" else V.BIN_NEAREST
    f0, df = H.lattice_of(tiny)
    st = V.Stack(tiny.nu, tiny.nv, tiny.nrest, tiny.npol, tiny.du, tiny.dv, rest_f0=f0, rest_df=df,
                 bin_mode=bin_mode)
    try:
        for s in tiny.spws:
            g_vis, g_w, g_uvw = st.regrid_rows(s.uvw, s.freqs, s.vis, s.flags, l=s.l, m=s.m, z=s.z, with_uvw=True)
            src = H.O.Source(s.uvw.cpu().numpy(), s.freqs, s.vis.cpu().numpy(), s.weights.cpu().numpy(),
                             s.flags.cpu().numpy(), s.l, s.m, s.z)
            o_vis, o_w = H.O.regrid_rows(src, f0, df, tiny.nrest, bin_mode)
            _check(g_vis, g_w, o_vis, o_w, float(s.vis.abs().max()))
            np.testing.assert_allclose(g_uvw.cpu().numpy(), s.uvw.cpu().numpy() / (1.0 + s.z), rtol=1e-15)
    finally:
        st.close()


def test_regrid_rows_half_storage(V, tiny):
    f0, df = H.lattice_of(tiny)
    st = V.Stack(tiny.nu, tiny.nv, tiny.nrest, tiny.npol, tiny.du, tiny.dv, rest_f0=f0, rest_df=df)
    try:
        s = tiny.spws[2]
        q, scale, deq = H.quantise(s.vis, "f16")
        g_vis, g_w, _ = st.regrid_rows(s.uvw, s.freqs, q, s.flags, l=s.l, m=s.m, z=s.z, vis_scale=scale)
        src = H.O.Source(s.uvw.cpu().numpy(), s.freqs, deq, s.weights.cpu().numpy(), s.flags.cpu().numpy(),
                         s.l, s.m, s.z)
        o_vis, o_w = H.O.regrid_rows(src, f0, df, tiny.nrest)
        _check(g_vis, g_w, o_vis, o_w, float(np.abs(deq).max()))
    finally:
        st.close()


def test_regrid_rows_needs_a_lattice(V, tiny):
    s = tiny.spws[0]
    st = V.Stack(tiny.nu, tiny.nv, tiny.nrest, tiny.npol, tiny.du, tiny.dv, central_freq=tiny.central_freq)
    try:
        with pytest.raises(V.VistaError) as ei:
            st.regrid_rows(s.uvw, s.freqs, s.vis, s.flags, l=s.l, m=s.m, z=s.z)
        assert ei.value.code == V.E_STATE
        for x in tiny.spws:
            st.add_source(x.uvw, x.freqs, x.vis, x.weights, x.flags, l=x.l, m=x.m, z=x.z)
        st.run()                                   # the run fixes the lattice
        g_vis, g_w, _ = st.regrid_rows(s.uvw, s.freqs, s.vis, s.flags, l=s.l, m=s.m, z=s.z)
        f0, df = st.lattice()
    finally:
        st.close()
    src = H.O.Source(s.uvw.cpu().numpy(), s.freqs, s.vis.cpu().numpy(), s.weights.cpu().numpy(),
                     s.flags.cpu().numpy(), s.l, s.m, s.z)
    o_vis, o_w = H.O.regrid_rows(src, f0, df, tiny.nrest)
    _check(g_vis, g_w, o_vis, o_w, float(s.vis.abs().max()))
