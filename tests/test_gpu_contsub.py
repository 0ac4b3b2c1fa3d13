"""Continuum subtraction over the rest axis (vista_contsub, the first
post-processing step of Sec. 3.4) against the oracle (oracle/contsub.py).

Two comparisons:
  * the kernel's arithmetic: GPU contsub of the GPU's cube against the
    oracle's fit applied to the same cube read back in FP64; and
  * end to end: GPU stack + GPU contsub against oracle stack + oracle fit,
    with the error scale of the stacking parity bound carried through the
    fit.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_01897_gb300 import build
    build.build()
    from paper_2609_01897_gb300 import vista
    vista.lib()
    return vista


def _stack(V, wl, precision):
    st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, rest_f0=wl.rest_f0, rest_df=wl.rest_df,
                 central_freq=wl.central_freq, precision=precision)
    for s in wl.spws:
        st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z, pol_map=s.pol_map)
    st.run()
    return st


def _line_free(nrest, seed):
    rng = np.random.default_rng(seed)
    free = rng.random(nrest) < 0.7
    free[nrest // 2 - 6: nrest // 2 + 6] = False     # the line's channels around the cube centre
    return free


def _kernel_check(got, wv, w, free, order):
    from oracle import contsub as CS
    want = CS.contsub(wv, w, free, order)
    g = got[..., 0].astype(np.float64) + 1j * got[..., 1].astype(np.float64)
    scale = np.abs(wv) + np.abs(wv - want)
    err = np.abs(g - want)
    bad = err > TOL * scale + 1e-30
    assert not bad.any(), "worst %.3g at %s" % (float((err / np.maximum(scale, 1e-300)).max()),
                                                 np.argwhere(bad)[0])
    return float((err[scale > 0] / scale[scale > 0]).max())


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_contsub_kernel_matches_oracle_fit(V, prec, order):
    from paper_2609_01897_gb300 import synth
    wl = synth.tiny("cuda")
    st = _stack(V, wl, V.PREC_MIXED if prec == "mixed" else V.PREC_FP64)
    try:
        cube = st.read_cube(device=True, f64=True)
        wv = (cube["sum_wv"][..., 0] + 1j * cube["sum_wv"][..., 1]).cpu().numpy()
        w = cube["sum_w"].cpu().numpy()
        free = _line_free(wl.nrest, order)
        got = st.contsub(free, order).cpu().numpy()
        # the cube itself is unchanged
        again = st.read_cube(device=True, f64=True)
        assert torch.equal(again["sum_wv"], cube["sum_wv"])
    finally:
        st.close()
    assert (w > 0).sum() > 1000
    _kernel_check(got, wv, w, free, order)


def test_contsub_end_to_end_against_oracle_stack(V):
    """GPU stack + contsub against oracle stack + oracle fit.  The stack's
    parity bound |d sum_wv| <= 1e-5 sum W w |V| (and 1e-5 relative on sum_w)
    carries through the linear fit: the fitted term of channel j moves by at
    most 1e-5 times sum_w_j times the weighted mean |V| of the fit set, up
    to the fit's leverage (a few for low orders), which the bound allows."""
    from oracle import contsub as CS
    from paper_2609_01897_gb300 import synth
    from tests import gpu_helpers as H
    wl = synth.tiny("cuda")
    o = H.run_oracle(wl)
    st = _stack(V, wl, V.PREC_MIXED)
    free = _line_free(wl.nrest, 11)
    try:
        got = st.contsub(free, 1).cpu().numpy()
    finally:
        st.close()
    want = CS.contsub(o["sum_wv"], o["sum_w"], free, 1)
    g = got[..., 0].astype(np.float64) + 1j * got[..., 1].astype(np.float64)
    fitset = free[None, None, :, None] & (o["sum_w"] > 0)
    mean_abs = (np.where(fitset, o["sum_wabs"], 0).sum(axis=2, keepdims=True) /
                np.maximum(np.where(fitset, o["sum_w"], 0).sum(axis=2, keepdims=True), 1e-300))
    scale = o["sum_wabs"] + o["sum_w"] * mean_abs * 8.0
    err = np.abs(g - want)
    assert (err <= TOL * scale + 1e-30).all(), float((err / np.maximum(scale, 1e-300)).max())


def test_contsub_host_destination_and_errors(V):
    from paper_2609_01897_gb300 import synth
    wl = synth.tiny("cuda")
    st = _stack(V, wl, V.PREC_MIXED)
    try:
        free = _line_free(wl.nrest, 3)
        dev = st.contsub(free, 2).cpu()
        host = st.contsub(free, 2, device=False)
        assert not host.is_cuda
        assert torch.equal(dev, host)
        L = V.lib()
        buf = torch.empty_like(dev)
        lf = np.ones(wl.nrest, dtype=np.uint8)
        assert L.vista_contsub(st.h, lf.ctypes.data, 4, buf.data_ptr(), 0) == V.E_ARG
        assert L.vista_contsub(st.h, lf.ctypes.data, -1, buf.data_ptr(), 0) == V.E_ARG
        assert L.vista_contsub(st.h, None, 1, buf.data_ptr(), 0) == V.E_ARG
        assert "order" in V.last_error(st.h) or "null" in V.last_error(st.h)
        # no line-free channel: nothing is subtracted
        none = st.contsub(np.zeros(wl.nrest, dtype=bool), 1).cpu()
        cube = st.read_cube(device=True)
        assert torch.equal(none, cube["sum_wv"].cpu())
    finally:
        st.close()


def test_contsub_removes_a_flat_continuum_from_stacked_data(V):
    """A point source with a flat spectrum, stacked and continuum-subtracted
    with order 0: every cell's line-free channels average to zero, and with
    no line in the data every channel is ~0 (the model is the data)."""
    import math
    from paper_2609_01897_gb300 import synth
    rng = np.random.default_rng(4)
    enu = synth.array_enu(10, 500.0, rng)
    uvw = synth.uvw_tracks(enu, -23.0, -30.0, 20, 30.0, 0.2)
    f = 230e9 + 15.625e6 * np.arange(64)
    l0, m0 = 3e-5, -2e-5
    u = torch.as_tensor(uvw, device="cuda")
    n1 = math.sqrt(1 - l0 * l0 - m0 * m0) - 1
    tau = (u[:, 0] * l0 + u[:, 1] * m0 + u[:, 2] * n1)[:, None] * torch.as_tensor(f, device="cuda")[None, :] / 299792458.0
    vis = (2.0 * torch.exp(-2j * math.pi * tau)).to(torch.complex64)[..., None].repeat(1, 1, 2).contiguous()
    w = torch.ones((uvw.shape[0], 2), dtype=torch.float32, device="cuda")
    spw = synth.SourceSpw(u, f, vis, w, None, l0, m0, 0.5)
    du = 2 * 1.001 * np.abs(uvw[:, :2]).max() * f.max() / 299792458.0 / 32
    wl = synth.Workload("flat", 32, 32, 48, 2, du, du, 230.5e9 * 1.5, [spw])
    st = _stack(V, wl, V.PREC_MIXED)
    try:
        cube = st.read_cube(device=True, f64=True)
        out = st.contsub(np.ones(wl.nrest, dtype=bool), 0).cpu().numpy()
    finally:
        st.close()
    sw = cube["sum_w"].cpu().numpy()
    swv = cube["sum_wv"].cpu().numpy()
    assert (sw > 0).sum() > 100
    # the stacked spectrum is 2 + 0i everywhere (the point source is real after the shift)
    np.testing.assert_allclose(swv[..., 0][sw > 0] / sw[sw > 0], 2.0, rtol=2e-5)
    assert np.abs(out[..., 0][sw > 0] / sw[sw > 0]).max() < 1e-4
    assert np.abs(out[..., 1][sw > 0] / sw[sw > 0]).max() < 1e-4


@pytest.mark.parametrize("planes", [1, 3, 4])
def test_contsub_kernel_other_plane_counts(V, planes):
    """Cubes of 1 and 4 planes (a warp per uv cell, lane L on plane L mod
    npol) and of 3 planes (a warp per cell and plane), against the oracle's
    fit on the same cube, orders 1 and 3."""
    from paper_2609_01897_gb300 import synth
    pols = {1: (1,), 3: (2,), 4: (4,)}[planes]
    wl = synth.random_case(57 + planes, "cuda", nsrc=5, max_rows=200, npol_choices=pols, nrest=64)
    wl.npol = planes      # three planes: the windows' two pols fill planes 0 and 1
    for order in (1, 3):
        st = _stack(V, wl, V.PREC_MIXED)
        try:
            cube = st.read_cube(device=True, f64=True)
            wv = (cube["sum_wv"][..., 0] + 1j * cube["sum_wv"][..., 1]).cpu().numpy()
            w = cube["sum_w"].cpu().numpy()
            free = _line_free(wl.nrest, order)
            got = st.contsub(free, order).cpu().numpy()
        finally:
            st.close()
        assert (w > 0).sum() > 100
        _kernel_check(got, wv, w, free, order)


@pytest.mark.parametrize("planes,nrest", [(1, 1024), (2, 512), (4, 256)])
def test_contsub_long_spectra(V, planes, nrest):
    """Cells of 1024 entries (1, 2 or 4 planes of 1024, 512 or 256 rest
    channels): against the oracle's fit on the same cube, orders 0-3, mixed
    and FP64 cubes, with a random line-free mask and with a fit set of six
    channels (the FP64 refit of quadratic and cubic planes)."""
    from paper_2609_01897_gb300 import synth
    pols = {1: (1,), 2: (2,), 4: (4,)}[planes]
    wl = synth.random_case(71 + planes, "cuda", nsrc=6, max_rows=200, npol_choices=pols, nrest=nrest)
    wl.npol = planes
    few = np.zeros(nrest, dtype=bool)
    few[np.linspace(nrest // 8, nrest - nrest // 8, 6).astype(int)] = True
    for prec in ("mixed", "fp64"):
        st = _stack(V, wl, V.PREC_MIXED if prec == "mixed" else V.PREC_FP64)
        try:
            cube = st.read_cube(device=True, f64=True)
            wv = (cube["sum_wv"][..., 0] + 1j * cube["sum_wv"][..., 1]).cpu().numpy()
            w = cube["sum_w"].cpu().numpy()
            assert (w > 0).sum() > 1000
            for order in range(4):
                for free in (_line_free(nrest, order), few):
                    got = st.contsub(free, order).cpu().numpy()
                    _kernel_check(got, wv, w, free, order)
        finally:
            st.close()
