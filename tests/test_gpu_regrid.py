"""The paper's per-row output (Eq. 3, vista_regrid_rows) against the oracle's
plain per-row products: every row of every tiny window, both binning modes,
16-bit storage, the rest-frame uvw, the state error before the lattice is
fixed, and a full 3840-channel, 4-pol window (wide as the batched stack's)
regridded onto rest bins 32 channels wide."""
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
    # the kernel: FP32 weights and sums of a few terms (~1e-7 relative) and a
    # phasor within 5e-7 rad; the oracle: FP64
    np.testing.assert_allclose(g_w, o_w, rtol=1e-6, atol=1e-7)
    err = np.abs(g_vis - o_vis)
    assert (err <= 2e-6 * (np.abs(o_vis) + vis_scale)).all(), float((err / (np.abs(o_vis) + vis_scale)).max())
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


def test_regrid_rows_full_wide_window(V):
    """A window as wide as the batched stack's widest (3840 channels over
    1.875 GHz, 4 pols, 2000 rows, 3 % flags, offset 8 arcsec) on a lattice of
    rest bins 32 channels wide, every row and bin against the oracle."""
    from paper_2609_01897_gb300 import synth
    rng = np.random.default_rng(12)
    nrow, nchan, npol = 2000, 3840, 4
    enu = synth.array_enu(30, 3000.0, rng)
    uvw = synth.uvw_tracks(enu, -23.0, -30.0, (nrow + 434) // 435, 30.0, 0.1)[:nrow]
    df_obs = 1.875e9 / nchan
    f = 380e9 + df_obs * np.arange(nchan)
    g = torch.Generator(device="cuda")
    g.manual_seed(12)
    vis = torch.complex(torch.randn((nrow, nchan, npol), generator=g, device="cuda"),
                        torch.randn((nrow, nchan, npol), generator=g, device="cuda")).to(torch.complex64)
    flags = (torch.rand((nrow, nchan, npol), generator=g, device="cuda") < 0.03).to(torch.uint8)
    u = torch.as_tensor(uvw, device="cuda")
    l0, m0, z = 8 * np.pi / 180 / 3600, -5 * np.pi / 180 / 3600, 1.7
    rest_df = 32 * df_obs * (1 + z)
    nrest = nchan // 32 + 4
    f0 = f[0] * (1 + z) - 2 * rest_df
    st = V.Stack(16, 16, nrest, npol, 1.0, 1.0, rest_f0=f0, rest_df=rest_df)
    try:
        g_vis, g_w, _ = st.regrid_rows(u, f, vis, flags, l=l0, m=m0, z=z)
    finally:
        st.close()
    src = H.O.Source(uvw, f, vis.cpu().numpy(), np.ones((nrow, npol), dtype=np.float32), flags.cpu().numpy(),
                     l0, m0, z)
    o_vis, o_w = H.O.regrid_rows(src, f0, rest_df, nrest)
    assert (o_w > 0).sum() > nrow * npol * (nchan // 32 - 2)
    _check(g_vis, g_w, o_vis, o_w, float(vis.abs().max()))


def test_regrid_rows_ragged_pols_axes_and_alignment(V):
    """Ragged windows (1, 2 and 4 pols, descending channel axes, odd channel
    counts; the vector-load path and the per-element path), one 2-pol window
    whose visibilities start 8 bytes past a 16-byte boundary (the
    per-element path), and 2- and 4-pol windows whose outputs start 4 bytes
    past a 16-byte boundary (the per-value stores), each against the
    oracle."""
    from paper_2609_01897_gb300 import synth
    wl = synth.random_case(41, "cuda", nsrc=6, max_rows=60, npol_choices=(1, 2, 4), descending=True)
    f0, df = H.lattice_of(wl)
    st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, rest_f0=f0, rest_df=df)
    checked, unaligned_out = 0, 0
    try:
        for s in wl.spws:
            if s.vis.shape[0] == 0:
                continue
            vis = s.vis
            if vis.shape[2] == 2 and checked % 2 == 0:
                buf = torch.empty(vis.numel() + 1, dtype=torch.complex64, device=vis.device)
                vis = buf[1:].view(vis.shape)
                vis.copy_(s.vis)
                assert vis.data_ptr() % 16 == 8
            out = None
            if vis.shape[2] in (2, 4) and checked % 2 == 1:
                shp = (vis.shape[0], wl.nrest, vis.shape[2])
                n = int(np.prod(shp))
                bo = torch.zeros(2 * n + 1, dtype=torch.float32, device=vis.device)
                bw = torch.zeros(n + 1, dtype=torch.float32, device=vis.device)
                out = (bo[1:].view(*shp, 2), bw[1:].view(shp))
                assert out[0].data_ptr() % 16 == 4 and out[1].data_ptr() % 8 == 4
                unaligned_out += 1
            g_vis, g_w, _ = st.regrid_rows(s.uvw, s.freqs, vis, s.flags, l=s.l, m=s.m, z=s.z, out=out)
            if out is not None:
                assert g_vis.data_ptr() == out[0].data_ptr() and g_w.data_ptr() == out[1].data_ptr()
                g_vis = torch.complex(g_vis[..., 0], g_vis[..., 1])
            src = H.O.Source(s.uvw.cpu().numpy(), s.freqs, s.vis.cpu().numpy(), s.weights.cpu().numpy(),
                             s.flags.cpu().numpy(), s.l, s.m, s.z)
            o_vis, o_w = H.O.regrid_rows(src, f0, df, wl.nrest)
            if (o_w > 0).any():
                _check(g_vis, g_w, o_vis, o_w, float(s.vis.abs().max()))
                checked += 1
    finally:
        st.close()
    assert checked >= 3 and unaligned_out >= 1, (checked, unaligned_out)
